"""Planted mistakes in the oracle (on the CPU) must fail the pins.

Each case patches one plausible error into a copy of an oracle step and checks
that the corresponding pin rejects it: a dropped factor, a wrong sign, a wrong
mass power, a transposed axis."""
import math
import numpy as np
import scipy.sparse as sp
from scipy.special import gammainc

import oracle
import synth
from oracle.chfsi import Bounds
from test_oracle_hamiltonian import one_d_operator, _nl_system
from test_oracle_chfsi import cheb_T, wells_system


def _kron_ref(L, n, p, m):
    Kt = [one_d_operator(L[d], n[d], p)[2] for d in range(3)]
    I = [np.eye(m.g[d]) for d in range(3)]
    return 0.5 * (np.kron(I[2], np.kron(I[1], Kt[0])) + np.kron(I[2], np.kron(Kt[1], I[0]))
                  + np.kron(Kt[2], np.kron(I[1], I[0])))


def test_dropped_half_in_stiffness_is_caught():
    L, n, p = (4.0, 5.0, 6.0), (2, 3, 2), 2
    m = oracle.PeriodicMesh(L, n, p)
    H = oracle.Hamiltonian(m)
    ref = _kron_ref(L, n, p, m)
    assert np.abs(H.dense() - ref).max() < 1e-12 * np.abs(ref).max()
    H.K = 2.0 * H.K
    H._Hc = None
    assert np.abs(H.dense() - ref).max() > 1e-3


def test_swapped_axes_in_stiffness_is_caught():
    L, n, p = (4.0, 5.0, 6.0), (2, 3, 2), 2
    m = oracle.PeriodicMesh(L, n, p)
    H = oracle.Hamiltonian(m)
    m.h = m.h[[1, 0, 2]]                      # x and y cell sizes swapped in the derivative scaling
    Hbad = oracle.Hamiltonian(m)
    ref = _kron_ref(L, n, p, m)
    assert np.abs(Hbad.dense() - ref).max() > 1e-3


def test_wrong_recurrence_sign_is_caught():
    m, H = wells_system(nl=True)
    lam, V = np.linalg.eigh(H.dense())
    bd = Bounds(a=lam[10], b=lam[-1] + 0.5)
    e, c = (bd.b - bd.a) / 2, (bd.b + bd.a) / 2

    def bad_filter(apply, X, degree, bounds):
        Y = (apply(X) - c * X) / e
        for _ in range(2, degree + 1):
            X, Y = Y, 2.0 * (apply(Y) - c * Y) / e + X        # planted: + X_{k-1}
        return Y
    t = cheb_T(7, (lam - c) / e)
    Y = bad_filter(H.apply, V[:, :4], 7, bd)
    assert np.abs(Y - V[:, :4] * t[:4]).max() > 1e-3 * max(1.0, np.abs(t).max())


def test_wrong_mass_power_in_projectors_is_caught():
    m, H, cent, (rowptr, node, chi, h) = _nl_system(ncell=4, p=6, L=9.0)
    cols = np.repeat(np.arange(h.size), np.diff(rowptr))
    bad = sp.csr_matrix((m.mass[node] * chi, (node, cols)), shape=(m.ndofs, h.size))   # M chi, not M^1/2 chi
    norms = np.asarray(bad.multiply(bad).sum(axis=0)).ravel()
    assert abs(norms[0] - gammainc(1.5, 9.0)) > 2e-2


def test_unscaled_potential_quadrature_weight_is_caught():
    m = oracle.PeriodicMesh((3.0, 4.0, 5.0), 2, 3)
    H = oracle.Hamiltonian(m, vquad=0)
    H.set_potential(np.full((m.ncells, H.nq), 1.3))
    H.Wq = np.ones_like(H.Wq)                 # planted: quadrature weights dropped
    assert abs(H.cell_V(0).sum() - 1.3 * np.prod(m.h)) > 1e-3


def test_density_without_mass_scaling_is_caught():
    """Planted: psi~ used at the quadrature points without the M^-1/2 back-transform."""
    from oracle.density import fermi_dirac, fermi_level, rayleigh_ritz_split, KB_HA_PER_K
    m, H = wells_system(nl=False, vquad=1)
    N, nfr = 12, 4
    lam, V = np.linalg.eigh(H.dense())
    X = V[:, :N]
    th_fr, Xfr, th = rayleigh_ritz_split(H.apply, X, nfr)
    kT = 500 * KB_HA_PER_K
    ne = 2 * (N - nfr) + 3.1
    f = fermi_dirac(th_fr, fermi_level(th_fr, N - nfr, ne, kT), kT)
    bad = np.empty((m.ncells, H.nq))
    for c in range(m.ncells):
        rows = m.cell_map[c]
        Po, Pf = H.Nq @ X[rows], H.Nq @ Xfr[rows]                 # missing M^-1/2
        bad[c] = 2.0 * (np.sum(Po * Po, axis=1) + (Pf * Pf) @ (f - 1.0))
    assert abs(np.sum(bad * (H.Wq * m.detJ)[None, :]) - ne) > 1e-2


# ---------------------------------------------------------------- Bloch k-points
def _kpoint_kron(L, n, p, k, m):
    from test_oracle_kpoint import one_d_bloch
    A = [one_d_bloch(L[d], n[d], p, k[d]) for d in range(3)]
    I = [np.eye(m.g[d]) for d in range(3)]
    return (np.kron(I[2], np.kron(I[1], A[0])) + np.kron(I[2], np.kron(A[1], I[0]))
            + np.kron(A[2], np.kron(I[1], I[0])))


def test_k_terms_mistakes_are_caught_by_the_kronecker_pin():
    """Dropping 1/2|k|^2, flipping the sign of the -i k.grad term (i.e. using +i) without
    flipping k elsewhere, or permuting k's components all move H~^k off the Kronecker sum of
    1D Bloch operators; the correct oracle is on it."""
    from oracle import kpoint
    L, n, p, k = (4.0, 5.0, 6.0), (2, 3, 2), 2, (0.3, -0.7, 0.2)
    m = oracle.PeriodicMesh(L, n, p)
    ref = _kpoint_kron(L, n, p, k, m)
    B = kpoint.BlochHamiltonian(oracle.Hamiltonian(m), k)
    assert np.abs(B.dense() - ref).max() < 1e-12 * np.abs(ref).max()
    Bk = B.Bk.copy()
    # Bk = -i k.G + 1/2|k|^2 M^c: its real part is the (diagonal) mass term
    assert np.abs(Bk.real - np.diag(Bk.real.diagonal())).max() == 0.0
    for name, bad in (("no 1/2|k|^2", Bk - np.diag(Bk.real.diagonal())),
                      ("+i k.grad", np.conj(Bk)),
                      ("permuted k", kpoint.BlochHamiltonian(oracle.Hamiltonian(m), (k[1], k[0], k[2])).Bk)):
        B.Bk = bad
        assert np.abs(B.dense() - ref).max() > 1e-3 * np.abs(ref).max(), name
