"""Spectrum splitting and electron density (oracle, FP64).

Alg. 2 with spectrum splitting: only the top N_fr eigenpairs of the projected problem
are used, Psi_fr = Psi_f Q_fr, together with the orthonormal basis Psi_o = Psi_f L^-T.
In the orthonormalise-first reading (CholGS gives X = Psi_o), Q_fr = L^-T Q'_fr and
Psi_fr = X Q'_fr, with Q'_fr the top N_fr eigenvectors of X^T H~ X.

Alg. 3: the Fermi level mu from 2 (N_oc + sum_fr f(eps_i, mu)) = N_e (the lowest
N_oc = N - N_fr states fully occupied; the paper's sum index is read as running over
the N_fr fractionally occupied states), then, with psi^ = M^-1/2 psi~,
rho(x) = 2 n(x)^T [Psi^_o Psi^_o^T + Psi^_fr (f(D_fr) - I) Psi^_fr^T] n(x)
at the quadrature points of each cell.  f is Fermi-Dirac, f = 1 / (1 + exp((eps - mu)/kT)).
"""
import numpy as np
from scipy.special import expit

from .chfsi import sign_fix

KB_HA_PER_K = 3.166811563e-6          # Boltzmann constant in Hartree per kelvin (CODATA 2018)


def fermi_dirac(eps, mu, kT):
    return expit(-(np.asarray(eps, np.float64) - mu) / kT)


def fermi_level(eps_fr, n_oc, n_elec, kT, iters=200):
    """mu with 2 (n_oc + sum_i f(eps_i, mu)) = n_elec, by bisection (the count is increasing in mu)."""
    eps_fr = np.asarray(eps_fr, np.float64)
    if not (2 * n_oc < n_elec < 2 * (n_oc + eps_fr.size)):
        raise ValueError("the electron count must fall inside the fractionally occupied window")
    lo, hi = eps_fr.min() - 50 * kT, eps_fr.max() + 50 * kT
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if 2.0 * (n_oc + fermi_dirac(eps_fr, mid, kT).sum()) < n_elec:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def rayleigh_ritz_split(apply, Xo, nfr):
    """Top-nfr Ritz pairs of the orthonormal basis Xo: (theta_fr ascending, Psi_fr = Xo Q'_fr)."""
    W = apply(Xo)
    Hh = Xo.T @ W
    Hh = 0.5 * (Hh + Hh.T)
    theta, Q = np.linalg.eigh(Hh)
    Q = sign_fix(Q)
    N = Xo.shape[1]
    return theta[N - nfr:], Xo @ Q[:, N - nfr:], theta


def density(ham, Xo, Xfr, f_fr, cells=None):
    """rho at the quadrature points of every cell (ncells x n_q), Alg. 3 formula; with
    `cells`, only those cells (len(cells) x n_q)."""
    m = ham.mesh
    s = 1.0 / np.sqrt(m.mass)
    cells = range(m.ncells) if cells is None else cells
    out = np.empty((len(cells), ham.nq))
    w = np.asarray(f_fr, np.float64) - 1.0
    for r, c in enumerate(cells):
        rows = m.cell_map[c]
        Po = ham.Nq @ (s[rows, None] * Xo[rows])           # psi^_o at the quadrature points
        Pf = ham.Nq @ (s[rows, None] * Xfr[rows])
        out[r] = 2.0 * (np.sum(Po * Po, axis=1) + (Pf * Pf) @ w)
    return out
