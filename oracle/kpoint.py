"""Bloch k-point Hamiltonian and the complex ChFSI steps (oracle, complex128).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With the Bloch form psi = e^{ik.x} u (Sec. 2.1, Eq. bloch), the periodic part u solves
the reduced Kohn-Sham equation on the cell (Sec. 2.1, the equation after Eq. bloch):
  (-1/2 lap - i k.grad + 1/2 |k|^2 + V_loc) u + e^{-ik.x} V_nl (e^{ik.y} u) = eps u.
Discretised with the same real spectral-element basis N_j and the same quadratures as at
the Gamma point (hamiltonian.py), cell by cell:
  H^{c,k}_jl = K^c_jl + V^c_jl - i sum_d k_d G^c_{d,jl} + 1/2 |k|^2 M^c_jl,
  G^c_{d,jl} = int_c N_j dN_l/dx_d      GLL quadrature on the nodes,
  M^c_jl     = int_c N_j N_l            GLL quadrature on the nodes (diagonal),
  H~^{c,k}  = D_c^-1/2 H^{c,k} D_c^-1/2 (D_c = global lumped M at the cell's nodes).
Nonlocal term: the coefficients C^{a,nk} of the paper's nonlocal energy are projections of u
on the Bloch sum of the projector, so the operator seen by u is sum_a h_a |g_a><g_a| with
  g_a(x) = sum_r chi_a(x - R_a - L_r) e^{-ik.(x - R_a - L_r)}
(a constant phase e^{-ik.R_a} dropped: it cancels in |g><g|).  With the projector cut off
inside half the box only the minimum-image displacement d = x - R_a - L_r contributes, and
GLL collocation gives C~^k_ja = M_jj^1/2 chi_a(d_j) e^{-ik.d_j}, H~_nl^k = C~^k diag(h) C~^k^H.

Complex blocks are M x N complex128; their real view (numpy .view(float64)) is the M x 2N
matrix whose columns interleave real and imaginary parts.

ChFSI steps for complex blocks (Eq. chebyfilter, Alg. 2 read as orthonormalise-first, as
in chfsi.py), with the Hermitian transpose in place of the transpose:
  filter:   chfsi.chebyshev_filter (real coefficients, complex vectors);
  CholGS:   S = X^H X = L L^H, X <- X L^-H;
  RR:       W = H~^k X, H^ = (X^H W + W^H X)/2 = Q Theta Q^H, X <- X Q, W <- W Q, each column
            of Q multiplied by the phase that makes its largest-|.| entry real and positive;
  residual: r_i = ||w_i - theta_i x_i||_2;
  bounds:   Lanczos (chfsi.lanczos_bounds) on the real 2M x 2M form of H~^k acting on the
            real view of one complex vector (the same spectrum, every eigenvalue twice).
"""
import math
import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_triangular

from .basis import lagrange_table, lagrange_deriv_table
from .chfsi import Bounds, chebyshev_filter, lanczos_bounds


class BlochHamiltonian:
    """H~^k for a Gamma-point Hamiltonian `ham` (potential set) and a wave vector k (bohr^-1)."""

    def __init__(self, ham, kvec):
        self.ham = ham
        self.mesh = m = ham.mesh
        self.k = np.asarray(kvec, np.float64).reshape(3).copy()
        n1 = m.n1
        lg = lagrange_table(m.xi, m.xi)            # N_j at the GLL nodes
        dg = lagrange_deriv_table(m.xi, m.xi)      # l_a' at the GLL nodes
        s = 2.0 / m.h
        Nn = np.einsum("ia,jb,kc->kjicba", lg, lg, lg).reshape(n1 ** 3, n1 ** 3)
        G = [s[0] * np.einsum("ia,jb,kc->kjicba", dg, lg, lg).reshape(n1 ** 3, n1 ** 3),
             s[1] * np.einsum("ia,jb,kc->kjicba", lg, dg, lg).reshape(n1 ** 3, n1 ** 3),
             s[2] * np.einsum("ia,jb,kc->kjicba", lg, lg, dg).reshape(n1 ** 3, n1 ** 3)]
        wg = np.einsum("k,j,i->kji", m.w, m.w, m.w).ravel() * m.detJ
        grad = sum(self.k[d] * np.einsum("q,qj,ql->jl", wg, Nn, G[d]) for d in range(3))
        mass = np.einsum("q,qj,ql->jl", wg, Nn, Nn)
        self.Bk = -1j * grad + 0.5 * float(self.k @ self.k) * mass   # k-dependent cell term
        self.Ct = None
        self.h = np.zeros(0)

    # ------------------------------------------------------------- nonlocal
    def set_nonlocal(self, h, rowptr, node, chi, disp):
        """CSR by projector as in Hamiltonian.set_nonlocal; disp[e] = x_node - R_a (minimum
        image) of entry e."""
        m = self.mesh
        h = np.asarray(h, np.float64)
        node = np.asarray(node, np.int64)
        cols = np.repeat(np.arange(h.size), np.diff(np.asarray(rowptr, np.int64)))
        phase = np.exp(-1j * (np.asarray(disp, np.float64).reshape(-1, 3) @ self.k))
        vals = np.sqrt(m.mass[node]) * np.asarray(chi, np.float64) * phase
        self.Ct = sp.csr_matrix((vals, (node, cols)), shape=(m.ndofs, h.size))
        self.h = h.copy()

    # ---------------------------------------------------------------- local
    def cell_matrices(self):
        m = self.mesh
        d = 1.0 / np.sqrt(m.mass[m.cell_map])
        return self.ham.cell_matrices() + d[:, :, None] * self.Bk[None] * d[:, None, :]

    def cell_matrix(self, c):
        d = 1.0 / np.sqrt(self.mesh.mass[self.mesh.cell_map[c]])
        return self.ham.cell_matrix(c) + d[:, None] * self.Bk * d[None, :]

    def apply(self, X):
        m = self.mesh
        X = np.asarray(X, np.complex128)
        squeeze = X.ndim == 1
        X2 = X.reshape(m.ndofs, -1)
        B = X2.shape[1]
        Xc = (m.Q @ X2).reshape(m.ncells, m.nodes_per_cell, B)           # extraction
        Yc = np.matmul(self.cell_matrices(), Xc)                           # cell products
        Y = m.QT @ Yc.reshape(-1, B)                                       # assembly
        if self.Ct is not None and self.h.size:
            P = self.h[:, None] * (self.Ct.conj().T @ X2)                  # h C~^H X
            Y = Y + self.Ct @ P
        return Y.ravel() if squeeze else Y

    def apply_real_view(self, v):
        """The real 2M x 2M form acting on the real view of one complex vector."""
        z = np.ascontiguousarray(v, np.float64).view(np.complex128)
        return np.ascontiguousarray(self.apply(z)).view(np.float64)

    def sparse(self):
        m = self.mesh
        blk = sp.block_diag([sp.csr_matrix(a) for a in self.cell_matrices()], format="csr")
        H = (m.QT @ blk @ m.Q).tocsr()
        if self.Ct is not None and self.h.size:
            H = H + (self.Ct @ sp.diags(self.h) @ self.Ct.conj().T).tocsr()
        return H

    def dense(self):
        return self.sparse().toarray()


# ------------------------------------------------------------ ChFSI steps
def cholgs(X):
    """S = X^H X = L L^H, X <- X L^-H."""
    X = np.asarray(X, np.complex128)
    S = X.conj().T @ X
    L = np.linalg.cholesky(S)
    return solve_triangular(L, X.conj().T, lower=True).conj().T, S, L


def phase_fix(Q):
    """Multiply each column by the phase that makes its largest-|.| entry (first on ties)
    real and positive."""
    idx = np.argmax(np.abs(Q), axis=0)
    piv = Q[idx, np.arange(Q.shape[1])]
    ph = np.where(np.abs(piv) > 0, np.conj(piv) / np.where(np.abs(piv) > 0, np.abs(piv), 1.0), 1.0)
    return Q * ph[None, :]


def rayleigh_ritz(apply, X):
    """W = H~^k X, H^ = (X^H W + W^H X)/2 = Q Theta Q^H (ascending), X <- X Q, W <- W Q."""
    X = np.asarray(X, np.complex128)
    W = apply(X)
    Hh = X.conj().T @ W
    Hh = 0.5 * (Hh + Hh.conj().T)
    theta, Q = np.linalg.eigh(Hh)
    Q = phase_fix(Q)
    return X @ Q, W @ Q, theta, Hh


def residuals(X, W, theta, mass=None):
    """||w_i - theta_i x_i||_2 for unit x_i, and with the lumped mass the generalised form
    ||H psi - theta M psi|| / ||psi||, psi = M^-1/2 x (chfsi.residuals with the modulus)."""
    R = W - X * theta[None, :]
    r = np.sqrt(np.sum((R * R.conj()).real, axis=0))
    if mass is None:
        return r
    m = np.asarray(mass)[:, None]
    num = np.sqrt(np.sum(m * (R * R.conj()).real, axis=0))
    den = np.sqrt(np.sum((X * X.conj()).real / m, axis=0))
    return r, num / den


def spectrum_bounds(bh, v0_real, k):
    """Lanczos on the real form of H~^k from the real view v0_real (length 2M)."""
    return lanczos_bounds(bh.apply_real_view, v0_real, k)


def chfsi_pass(bh, X, block, degree, bounds):
    """One pass on a complex block: filter each column block, CholGS, RR, residuals, then
    the bounds update a <- theta_N, a0 <- theta_1 (b kept), as chfsi.chfsi_pass."""
    X = np.array(X, dtype=np.complex128, copy=True)
    N = X.shape[1]
    for j0 in range(0, N, block):
        j1 = min(N, j0 + block)
        X[:, j0:j1] = chebyshev_filter(bh.apply, X[:, j0:j1], degree, bounds)
    X, _, _ = cholgs(X)
    X, W, theta, _ = rayleigh_ritz(bh.apply, X)
    r = residuals(X, W, theta)
    nb = Bounds(a=float(theta[-1]), b=bounds.b,
                a0=bounds.a0 if math.isnan(bounds.a0) else float(theta[0]))
    return X, W, theta, r, nb
