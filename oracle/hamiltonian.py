"""Löwdin-transformed FE Hamiltonian and its action (oracle, FP64).

H~ = M^-1/2 H M^-1/2 (Eq. hep), with H = H^loc + H^nl (Eq. discreteHam,
Eq. nonlocalHamDiscrete) at the Gamma point, without the GGA term.

Cell matrices (Sec. 4.2 / Eq. celldgemm):
  K^c_jk = 1/2 sum_q w_q detJ grad N_j(x_q) . grad N_k(x_q)    GLL quadrature on the nodes
  V^c_jk = sum_q w_q detJ V(x_q) N_j(x_q) N_k(x_q)             Eq. quadLocal (Gauss p+1 or GLL)
  H~^c   = D_c^-1/2 (K^c + V^c) D_c^-1/2,  D_c = global lumped M at the cell's nodes
Local action (Eq. celldgemm): Y = ASEMB_FEM{ H~^c X^c } with X^c the gathered rows.
Nonlocal action (Alg. 4, Eq. nonlocalHamDiscrete): C_ja = int chi_a N_j ~= M_jj chi_a(x_j)
with GLL collocation, C~ = M^-1/2 C = M^1/2 chi, and Y += C~ diag(h) C~^T X.
"""
import numpy as np
import scipy.sparse as sp

from .basis import lagrange_table, lagrange_deriv_table


class Hamiltonian:
    def __init__(self, mesh, vquad=0):
        self.mesh = mesh
        self.vquad = int(vquad)
        m = mesh
        n1 = m.n1
        # basis at the potential quadrature points: Nq[q, j] = l_a(xa_q) l_b(xb_q) l_c(xc_q)
        xq, wq = m.quad_rule(self.vquad)
        nq = xq.size
        l = lagrange_table(m.xi, xq)
        self.Nq = np.einsum("ia,jb,kc->kjicba", l, l, l).reshape(nq ** 3, n1 ** 3)
        self.Wq = np.einsum("k,j,i->kji", wq, wq, wq).ravel()
        self.nq = nq ** 3
        # stiffness by GLL quadrature on the nodes (the definition, point by point)
        lg = lagrange_table(m.xi, m.xi)
        dg = lagrange_deriv_table(m.xi, m.xi)
        s = 2.0 / m.h
        Gx = s[0] * np.einsum("ia,jb,kc->kjicba", dg, lg, lg).reshape(n1 ** 3, n1 ** 3)
        Gy = s[1] * np.einsum("ia,jb,kc->kjicba", lg, dg, lg).reshape(n1 ** 3, n1 ** 3)
        Gz = s[2] * np.einsum("ia,jb,kc->kjicba", lg, lg, dg).reshape(n1 ** 3, n1 ** 3)
        wg = np.einsum("k,j,i->kji", m.w, m.w, m.w).ravel() * m.detJ
        self.K = 0.5 * (np.einsum("q,qj,qk->jk", wg, Gx, Gx)
                        + np.einsum("q,qj,qk->jk", wg, Gy, Gy)
                        + np.einsum("q,qj,qk->jk", wg, Gz, Gz))
        self.v_quad = np.zeros((m.ncells, self.nq))
        self.Ct = None
        self.h = np.zeros(0)
        self._Hc = None

    # ---------------------------------------------------------------- local
    def set_potential(self, v_quad):
        v = np.asarray(v_quad, np.float64).reshape(self.mesh.ncells, self.nq)
        self.v_quad = v.copy()
        self._Hc = None

    def cell_V(self, c):
        """V^c_jk = sum_q (w_q detJ V(x_q)) N_j(x_q) N_k(x_q), as Nq^T diag(w detJ V) Nq."""
        wv = self.Wq * self.mesh.detJ * self.v_quad[c]
        return (self.Nq.T * wv[None, :]) @ self.Nq

    def cell_matrix(self, c):
        d = 1.0 / np.sqrt(self.mesh.mass[self.mesh.cell_map[c]])
        return d[:, None] * (self.K + self.cell_V(c)) * d[None, :]

    def cell_matrices(self):
        if self._Hc is None:
            m = self.mesh
            wv = self.Wq[None, :] * m.detJ * self.v_quad
            V = np.matmul(self.Nq.T[None, :, :] * wv[:, None, :], self.Nq[None, :, :])
            d = 1.0 / np.sqrt(m.mass[m.cell_map])
            self._Hc = d[:, :, None] * (self.K[None] + V) * d[:, None, :]
        return self._Hc

    def apply_local(self, X):
        m = self.mesh
        X = np.asarray(X, np.float64)
        squeeze = X.ndim == 1
        X2 = X.reshape(m.ndofs, -1)
        B = X2.shape[1]
        Xc = (m.Q @ X2).reshape(m.ncells, m.nodes_per_cell, B)          # extraction
        Yc = np.matmul(self.cell_matrices(), Xc)                          # cell GEMMs
        Y = m.QT @ Yc.reshape(-1, B)                                      # ASEMB_FEM
        return Y.ravel() if squeeze else Y

    def _slots_of(self, rows):
        m = self.mesh
        flat = m.cell_map.ravel()
        order = np.argsort(flat, kind="stable")
        starts = np.searchsorted(flat[order], rows, side="left")
        ends = np.searchsorted(flat[order], rows, side="right")
        return [order[s:e] for s, e in zip(starts, ends)]

    def apply_local_rows(self, X, rows):
        """Rows `rows` of H~_loc X, computed cell by cell (for large meshes)."""
        m = self.mesh
        X2 = np.asarray(X).reshape(m.ndofs, -1)
        out = np.zeros((len(rows), X2.shape[1]))
        cache = {}
        for r, slots in enumerate(self._slots_of(np.asarray(rows))):
            for s in slots:
                c, l = divmod(int(s), m.nodes_per_cell)
                if c not in cache:
                    cache[c] = self.cell_matrix(c)
                out[r] += cache[c][l] @ X2[m.cell_map[c]]
        return out

    # ------------------------------------------------------------- nonlocal
    def set_nonlocal(self, h, rowptr, node, chi):
        m = self.mesh
        h = np.asarray(h, np.float64)
        rowptr = np.asarray(rowptr, np.int64)
        node = np.asarray(node, np.int64)
        chi = np.asarray(chi, np.float64)
        nproj = h.size
        cols = np.repeat(np.arange(nproj), np.diff(rowptr))
        vals = np.sqrt(m.mass[node]) * chi                                # C~ = M^1/2 chi
        self.Ct = sp.csr_matrix((vals, (node, cols)), shape=(m.ndofs, nproj))
        self.h = h.copy()

    def apply_nonlocal(self, X):
        if self.Ct is None or self.h.size == 0:
            return np.zeros_like(np.asarray(X, np.float64))
        X = np.asarray(X, np.float64)
        squeeze = X.ndim == 1
        X2 = X.reshape(self.mesh.ndofs, -1)
        P = self.Ct.T @ X2                       # projector coefficients (ASEMB_NLP)
        P = self.h[:, None] * P                  # scaling by h
        Y = self.Ct @ P                          # back to nodes (ASEMB_FEM)
        return Y.ravel() if squeeze else Y

    def apply_nonlocal_rows(self, X, rows):
        if self.Ct is None or self.h.size == 0:
            return np.zeros((len(rows), np.asarray(X).reshape(self.mesh.ndofs, -1).shape[1]))
        X2 = np.asarray(X).reshape(self.mesh.ndofs, -1)
        P = self.h[:, None] * (self.Ct.T @ X2)
        return self.Ct[np.asarray(rows)] @ P

    # ---------------------------------------------------------------- total
    def apply(self, X):
        return self.apply_local(X) + self.apply_nonlocal(X)

    def apply_rows(self, X, rows):
        return self.apply_local_rows(X, rows) + self.apply_nonlocal_rows(X, rows)

    def dense(self):
        """Assembled M x M H~ (tiny meshes only)."""
        m = self.mesh
        Hc = self.cell_matrices()
        blk = sp.block_diag([sp.csr_matrix(a) for a in Hc], format="csr")
        H = (m.QT @ blk @ m.Q).toarray()
        if self.Ct is not None and self.h.size:
            C = self.Ct.toarray()
            H += C @ np.diag(self.h) @ C.T
        return H

    def sparse(self):
        """Assembled sparse H~ (moderate meshes)."""
        m = self.mesh
        blk = sp.block_diag([sp.csr_matrix(a) for a in self.cell_matrices()], format="csr")
        H = (m.QT @ blk @ m.Q).tocsr()
        if self.Ct is not None and self.h.size:
            H = H + (self.Ct @ sp.diags(self.h) @ self.Ct.T).tocsr()
        return H
