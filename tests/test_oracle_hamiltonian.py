"""Oracle pins for H~ = M^-1/2 (K + V + C h C^T) M^-1/2 (Eq. discreteHam, Eq. hep,
Eq. nonlocalHamDiscrete).  Each pin uses an independent route to the answer:
1D assembly + Kronecker products, closed-form spectra, quadrature exactness."""
import os
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla
from scipy.special import gammainc

import oracle
import synth
from oracle.basis import gll_rule, gauss_rule, lagrange_table, lagrange_deriv_table

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def one_d_operator(L, n, p):
    """Independent 1D periodic GLL stiffness K1 and lumped mass M1, and K~1 = M1^-1/2 K1 M1^-1/2."""
    x, w = gll_rule(p)
    D = lagrange_deriv_table(x, x)
    h = L / n
    kloc = (2.0 / h) * (D.T * w) @ D           # int l_a' l_b' dx on one element
    g = n * p
    K1 = np.zeros((g, g))
    M1 = np.zeros(g)
    for c in range(n):
        idx = [(c * p + a) % g for a in range(p + 1)]
        K1[np.ix_(idx, idx)] += kloc
        M1[idx] += w * h / 2
    s = 1.0 / np.sqrt(M1)
    return K1, M1, s[:, None] * K1 * s[None, :]


def test_stiffness_annihilates_constants_and_is_psd():
    m = oracle.PeriodicMesh(5.0, 2, 4)
    H = oracle.Hamiltonian(m)
    assert np.abs(H.K @ np.ones(H.K.shape[0])).max() < 1e-12
    assert np.abs(H.K - H.K.T).max() < 1e-13
    assert np.linalg.eigvalsh(H.K).min() > -1e-12
    # the assembled operator annihilates M^1/2 * 1 (K . 1 = 0 globally)
    y = H.apply(np.sqrt(m.mass))
    assert np.abs(y).max() < 1e-11


@pytest.mark.parametrize("p,n,L", [(2, (2, 3, 2), (4.0, 5.0, 6.0)), (4, (3, 2, 2), (6.0, 6.0, 7.0))])
def test_free_electron_is_kronecker_sum(p, n, L):
    """V = 0: H~ = 1/2 (I (x) I (x) K~x + I (x) K~y (x) I + K~z (x) I (x) I) exactly (x fastest)."""
    m = oracle.PeriodicMesh(L, n, p)
    H = oracle.Hamiltonian(m)
    Kt = [one_d_operator(L[d], n[d], p)[2] for d in range(3)]
    I = [np.eye(m.g[d]) for d in range(3)]
    ref = 0.5 * (np.kron(I[2], np.kron(I[1], Kt[0])) + np.kron(I[2], np.kron(Kt[1], I[0]))
                 + np.kron(Kt[2], np.kron(I[1], I[0])))
    Hd = H.dense()
    assert np.abs(Hd - ref).max() < 1e-12 * np.abs(ref).max()
    # and the cell-by-cell action agrees with the dense matrix on a random block
    X = synth.random_block(3, m.ndofs, 5)
    assert np.abs(H.apply(X) - ref @ X).max() < 1e-12 * np.abs(ref).max()


def test_free_electron_converges_to_plane_waves():
    """Lowest 1D eigenvalues of K~1 -> (2 pi k / L)^2; 3D levels -> 1/2 |G|^2."""
    L = 10.0
    errs = []
    for p in (3, 5, 7):
        mu = np.linalg.eigvalsh(one_d_operator(L, 4, p)[2])
        exact = np.sort(np.array([(2 * np.pi * k / L) ** 2 for k in (0, 1, -1, 2, -2)]))
        errs.append(np.abs(mu[:5] - exact).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-7
    # 3D: the lowest 3D eigenvalues of the oracle's H~ are half-sums of the 1D ones
    m = oracle.PeriodicMesh(L, 2, 4)
    lam = np.linalg.eigvalsh(oracle.Hamiltonian(m).dense())[:27]
    mu = np.linalg.eigvalsh(one_d_operator(L, 2, 4)[2])
    sums = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel())[:27] / 2
    assert np.abs(lam - sums).max() < 1e-11
    assert abs(lam[1] - 0.5 * (2 * np.pi / L) ** 2) < 1e-2


def test_gll_collocated_constant_potential_is_a_shift():
    m = oracle.PeriodicMesh(6.0, 2, 3)
    H0 = oracle.Hamiltonian(m, vquad=1)
    H1 = oracle.Hamiltonian(m, vquad=1)
    H1.set_potential(np.full((m.ncells, H1.nq), -0.7))
    assert np.abs(H1.dense() - (H0.dense() - 0.7 * np.eye(m.ndofs))).max() < 1e-12


def test_gll_collocated_potential_is_diagonal_of_values():
    """vquad=1: the V term of H~ is diag(V(x_j)) (M^-1/2 (M V) M^-1/2)."""
    m = oracle.PeriodicMesh(6.0, 2, 3)
    H0 = oracle.Hamiltonian(m, vquad=1)
    H1 = oracle.Hamiltonian(m, vquad=1)
    q = m.quad_xyz(1).reshape(-1, 3)
    v = synth.gaussian_wells(q, [[1.0, 2.0, 3.0]], 2.0, 1.0, 6.0)
    H1.set_potential(v)
    vn = synth.gaussian_wells(m.node_xyz(), [[1.0, 2.0, 3.0]], 2.0, 1.0, 6.0)
    assert np.abs(H1.dense() - H0.dense() - np.diag(vn)).max() < 1e-12


@pytest.mark.parametrize("p", [1, 3, 5])
def test_gauss_constant_potential_is_consistent_mass(p):
    """vquad=0, V = v0: V^c = v0 * (1D consistent mass)^(x)3, the exact int N_j N_k."""
    m = oracle.PeriodicMesh((3.0, 4.0, 5.0), 2, p)
    H = oracle.Hamiltonian(m, vquad=0)
    H.set_potential(np.full((m.ncells, H.nq), 1.3))
    V = H.cell_V(0)
    x, _ = gll_rule(p)
    xg, wg = gauss_rule(2 * p + 4)            # an independent, higher-order rule
    T = lagrange_table(x, xg)
    mc = [(m.h[d] / 2) * (T.T * wg) @ T for d in range(3)]
    ref = 1.3 * np.kron(mc[2], np.kron(mc[1], mc[0]))
    assert np.abs(V - ref).max() < 1e-13
    assert abs(V.sum() - 1.3 * np.prod(m.h)) < 1e-12
    if p == 1:
        assert np.allclose(mc[0], m.h[0] / 6 * np.array([[2, 1], [1, 2]]), atol=1e-15)


def _lowest(H, k):
    A = H.sparse()
    return np.sort(spla.eigsh(A, k=k, sigma=-1.0, which="LM", return_eigenvectors=False))


@pytest.mark.slow
def test_harmonic_oscillator_levels_converge():
    ref = np.loadtxt(os.path.join(GOLD, "harmonic_levels.txt"))
    levels = np.repeat(ref[:, 0], ref[:, 1].astype(int))[:10]
    errs = []
    for p in (2, 3, 4, 5):
        m = oracle.PeriodicMesh(10.0, 4, p)
        H = oracle.Hamiltonian(m, vquad=0)
        H.set_potential(synth.harmonic(m.quad_xyz(0).reshape(-1, 3), (5.0, 5.0, 5.0), 1.0, 10.0))
        lam = _lowest(H, 10)
        errs.append(np.abs(lam - levels).max())
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-2
    assert abs(lam[0] - 1.5) < 5e-4 and np.abs(lam[1:4] - 2.5).max() < 1e-3


def _nl_system(seed=0, ncell=3, p=3, L=9.0):
    m = oracle.PeriodicMesh(L, ncell, p)
    H = oracle.Hamiltonian(m)
    xyz = m.node_xyz()
    cent = [[2.0, 3.0, 4.0], [6.5, 6.0, 5.5]]
    rowptr, node, chi = synth.projector_csr(xyz, cent, 1.0, 3.0, L)
    h = 0.5 + 1.5 * np.abs(synth.counter_uniform(seed, rowptr.size - 1))
    H.set_nonlocal(h, rowptr, node, chi)
    return m, H, cent, (rowptr, node, chi, h)


def test_nonlocal_psd_rank_and_locality():
    m, H, cent, (rowptr, node, chi, h) = _nl_system()
    C = H.Ct.toarray()
    Hnl = C @ np.diag(h) @ C.T
    ev = np.linalg.eigvalsh(Hnl)
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(ev > 1e-10 * ev.max()) <= h.size
    # zero on vectors supported away from both atoms
    X = np.zeros((m.ndofs, 2))
    far = np.setdiff1d(np.arange(m.ndofs), node)
    X[far, 0] = 1.0
    X[far[::3], 1] = -2.0
    assert np.abs(H.apply_nonlocal(X)).max() == 0.0
    # against the defining sum over projectors (Eq. nonlocalHamDiscrete, GLL collocation C = M chi)
    Y = H.apply_nonlocal(synth.random_block(2, m.ndofs, 3))
    ref = np.zeros_like(Y)
    Xr = synth.random_block(2, m.ndofs, 3)
    for a in range(h.size):
        nd = node[rowptr[a]:rowptr[a + 1]]
        Cja = m.mass[nd] * chi[rowptr[a]:rowptr[a + 1]]          # C_ja = M_jj chi_a(x_j)
        Ca = np.zeros(m.ndofs)
        Ca[nd] = Cja
        Ca_t = Ca / np.sqrt(m.mass)                               # M^-1/2 C
        ref += h[a] * np.outer(Ca_t, Ca_t @ Xr)
    assert np.abs(Y - ref).max() < 1e-12 * np.abs(ref).max()


def test_nonlocal_normalisation_by_quadrature():
    """C~_a^T C~_a = sum_j M_jj chi_a(x_j)^2 ~= int_{r<rc} chi_a^2 = P(3/2, rc^2/w^2) (s),
    P(5/2, rc^2/w^2) (p): regularised incomplete gamma (radial density r^2 e^-r^2 / r^4 e^-r^2)."""
    m, H, cent, (rowptr, node, chi, h) = _nl_system(ncell=4, p=6, L=9.0)
    C = H.Ct.toarray()
    norms = np.sum(C * C, axis=0)
    s_ref, p_ref = gammainc(1.5, 9.0), gammainc(2.5, 9.0)
    for a in range(2):
        assert abs(norms[4 * a] - s_ref) < 2e-2
        for mm in range(1, 4):
            assert abs(norms[4 * a + mm] - p_ref) < 2e-2


def test_nonlocal_weyl_monotonicity():
    m, H, cent, _ = _nl_system(ncell=2, p=3, L=9.0)
    Hl = oracle.Hamiltonian(m)
    ev_nl = np.linalg.eigvalsh(H.dense())
    ev_0 = np.linalg.eigvalsh(Hl.dense())
    assert np.all(ev_nl >= ev_0 - 1e-10)
    assert np.any(ev_nl > ev_0 + 1e-3)


def test_rows_match_full_application():
    m, H, cent, _ = _nl_system(ncell=3, p=2, L=9.0)
    q = m.quad_xyz(0).reshape(-1, 3)
    H.set_potential(synth.gaussian_wells(q, cent, 2.0, 1.0, 9.0))
    X = synth.random_block(5, m.ndofs, 4)
    rows = np.array([0, 1, 7, 100, m.ndofs - 1])
    assert np.abs(H.apply(X)[rows] - H.apply_rows(X, rows)).max() < 1e-12
