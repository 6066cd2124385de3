"""Periodic hexahedral spectral-element mesh (oracle, FP64).

Numbering (the paper is silent; the convention used here and by the library):
  global node (ix, iy, iz), ix in [0, nx*p), index = ix + gx*(iy + gy*iz), gx = nx*p;
  cell (cx, cy, cz) index = cx + nx*(cy + ny*cz);
  cell-local node (a, b, c) -> a + (p+1)*(b + (p+1)*c), global ix = (cx*p + a) mod gx;
  quadrature points in the same tensor order, x fastest.
Geometry: uniform cells of size h = L/n per axis, x = cx*h + (xi + 1)*h/2.
Lumped mass (Sec. 2.3, text after Eq. hep): M_jj = sum over cells containing j of
w_a w_b w_c * det J, with GLL weights w and det J = hx*hy*hz/8.
"""
import numpy as np
import scipy.sparse as sp

from .basis import gll_rule, gauss_rule


class PeriodicMesh:
    def __init__(self, L, ncell, degree, nq1d=None):
        self.L = np.broadcast_to(np.asarray(L, np.float64), (3,)).copy()
        self.n = np.broadcast_to(np.asarray(ncell, np.int64), (3,)).copy()
        if np.any(self.n < 2):
            raise ValueError("a periodic axis needs at least 2 cells")
        self.p = int(degree)
        self.nq1d = int(nq1d) if nq1d is not None else self.p + 1
        self.h = self.L / self.n
        self.g = self.n * self.p                       # nodes per axis
        self.ndofs = int(np.prod(self.g))
        self.ncells = int(np.prod(self.n))
        self.n1 = self.p + 1
        self.nodes_per_cell = self.n1 ** 3
        self.xi, self.w = gll_rule(self.p)
        self.detJ = float(np.prod(self.h)) / 8.0
        self._build_map()
        self._build_mass()

    def cell_coords(self, c):
        cx = c % self.n[0]
        cy = (c // self.n[0]) % self.n[1]
        cz = c // (self.n[0] * self.n[1])
        return cx, cy, cz

    def _build_map(self):
        n1, p = self.n1, self.p
        cmap = np.empty((self.ncells, self.nodes_per_cell), dtype=np.int64)
        a = np.arange(n1)
        A = np.tile(a, n1 * n1)
        B = np.tile(np.repeat(a, n1), n1)
        C = np.repeat(a, n1 * n1)
        for c in range(self.ncells):
            cx, cy, cz = self.cell_coords(c)
            ix = (cx * p + A) % self.g[0]
            iy = (cy * p + B) % self.g[1]
            iz = (cz * p + C) % self.g[2]
            cmap[c] = ix + self.g[0] * (iy + self.g[1] * iz)
        self.cell_map = cmap
        # Q: (ncells*n_c) x M selection matrix; gather = Q X, assembly = Q^T Y^c
        rows = np.arange(cmap.size)
        self.Q = sp.csr_matrix((np.ones(cmap.size), (rows, cmap.ravel())),
                               shape=(cmap.size, self.ndofs))
        self.QT = self.Q.T.tocsr()

    def _build_mass(self):
        w3 = np.einsum("c,b,a->cba", self.w, self.w, self.w).ravel() * self.detJ
        contrib = np.tile(w3, self.ncells)
        self.mass = self.QT @ contrib          # sum over cells of the cell's GLL weight
        self.cell_weights = w3

    def node_xyz(self):
        """Coordinates of all global nodes (M x 3)."""
        idx = np.arange(self.ndofs)
        ix = idx % self.g[0]
        iy = (idx // self.g[0]) % self.g[1]
        iz = idx // (self.g[0] * self.g[1])
        out = np.empty((self.ndofs, 3))
        for d, i in enumerate((ix, iy, iz)):
            cell = i // self.p
            a = i % self.p
            out[:, d] = cell * self.h[d] + (self.xi[a] + 1.0) * self.h[d] / 2.0
        return out

    def quad_rule(self, vquad=0):
        """1D rule for the local-potential term: Gauss (vquad=0) or GLL (vquad=1)."""
        if vquad == 1:
            return self.xi, self.w
        return gauss_rule(self.nq1d)

    def quad_xyz(self, vquad=0):
        """Quadrature point coordinates per cell (ncells x n_q x 3), tensor order x fastest."""
        xq, _ = self.quad_rule(vquad)
        nq = xq.size
        out = np.empty((self.ncells, nq ** 3, 3))
        QA = np.tile(np.arange(nq), nq * nq)
        QB = np.tile(np.repeat(np.arange(nq), nq), nq)
        QC = np.repeat(np.arange(nq), nq * nq)
        for c in range(self.ncells):
            cc = self.cell_coords(c)
            for d, qi in enumerate((QA, QB, QC)):
                out[c, :, d] = cc[d] * self.h[d] + (xq[qi] + 1.0) * self.h[d] / 2.0
        return out
