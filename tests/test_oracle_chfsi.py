"""Oracle pins for the ChFSI steps (Eq. chebyfilter, Alg. 2) against closed forms,
invariants and a dense eigensolve."""
import math
import numpy as np
import pytest

import oracle
import synth
from oracle.chfsi import (Bounds, chebyshev_filter, lanczos_bounds, cholgs, rayleigh_ritz,
                          rrgep_alg2, residuals, chfsi_pass, first_pass_bounds)


def cheb_T(m, x):
    """T_m(x) from its closed form: cos(m acos x) on [-1,1], sign^m cosh(m acosh|x|) outside."""
    x = np.asarray(x, np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


def wells_system(ncell=2, p=3, L=6.0, seed=0, nl=False, vquad=0):
    m = oracle.PeriodicMesh(L, ncell, p)
    H = oracle.Hamiltonian(m, vquad=vquad)
    s = synth.Stream(seed)
    cent = [[L * s.uniform() for _ in range(3)] for _ in range(3)]
    H.set_potential(synth.gaussian_wells(m.quad_xyz(vquad).reshape(-1, 3), cent, 2.0, 1.0, L))
    if nl:
        rowptr, node, chi = synth.projector_csr(m.node_xyz(), cent[:1], 1.0, 2.0, L)
        H.set_nonlocal(np.array([1.0, 0.7, 1.3, 0.9]), rowptr, node, chi)
    return m, H


@pytest.mark.parametrize("scaled", [False, True])
def test_filter_scalar_identity_on_eigenvectors(scaled):
    m, H = wells_system(nl=True)
    lam, V = np.linalg.eigh(H.dense())
    bd = Bounds(a=lam[10], b=lam[-1] + 0.5, a0=lam[0] - 0.1 if scaled else math.nan)
    deg = 9
    e, c = (bd.b - bd.a) / 2, (bd.b + bd.a) / 2
    t = cheb_T(deg, (lam - c) / e)
    if scaled:
        t = t / cheb_T(deg, np.array([(bd.a0 - c) / e]))[0]
    cols = [0, 3, 10, 50, len(lam) - 1]
    Y = chebyshev_filter(H.apply, V[:, cols], deg, bd)
    ref = V[:, cols] * t[cols][None, :]
    assert np.abs(Y - ref).max() < 1e-11 * max(1.0, np.abs(t).max())


def test_filter_degree_zero_and_one():
    m, H = wells_system()
    X = synth.random_block(1, m.ndofs, 3)
    bd = Bounds(a=1.0, b=50.0)
    assert np.array_equal(chebyshev_filter(H.apply, X, 0, bd), X)
    assert np.allclose(chebyshev_filter(H.apply, X, 1, bd), (H.apply(X) - 25.5 * X) / 24.5, atol=1e-13)


def test_lanczos_bounds_bracket_spectrum():
    m, H = wells_system(nl=True)
    lam = np.linalg.eigvalsh(H.dense())
    tmin, tmax, b = lanczos_bounds(H.apply, synth.counter_uniform(11, m.ndofs), 20)
    assert b >= lam[-1] - 1e-9
    Hd = H.dense()
    gersh = np.max(np.diag(Hd) + np.sum(np.abs(Hd), axis=1) - np.abs(np.diag(Hd)))
    assert b <= gersh
    assert tmin >= lam[0] - 1e-10 and tmax <= lam[-1] + 1e-10
    # b - lambda_max <= |beta_k| <= (lambda_max - lambda_min) / 2: every Lanczos coefficient
    # beta_j = v_{j+1}^T (H - c) v_j (v_{j+1} orthogonal to v_j) is at most ||H - c|| with c
    # the middle of the spectrum
    assert b - lam[-1] <= 0.5 * (lam[-1] - lam[0]) + 1e-9


def test_cholgs_orthonormal_and_span():
    m, H = wells_system()
    X = synth.random_block(2, m.ndofs, 12) @ np.diag(np.linspace(1, 100, 12))
    Xo, S, L = cholgs(X)
    assert np.abs(Xo.T @ Xo - np.eye(12)).max() < 1e-13
    P0 = X @ np.linalg.solve(X.T @ X, X.T)
    P1 = Xo @ Xo.T
    assert np.abs(P0 - P1).max() < 1e-12
    assert np.allclose(L @ L.T, X.T @ X, rtol=1e-13)
    assert np.allclose(np.tril(L), L)


def test_cholgs_rejects_rank_deficient():
    X = synth.random_block(3, 50, 4)
    X[:, 3] = X[:, 0]
    with pytest.raises(np.linalg.LinAlgError):
        cholgs(X)


def test_cholgs_rr_equals_alg2():
    m, H = wells_system(nl=True)
    X = synth.random_block(4, m.ndofs, 10)
    bd = Bounds(a=5.0, b=120.0, a0=-1.0)
    Psi = chebyshev_filter(H.apply, X, 6, bd)
    ref = rrgep_alg2(H.apply, Psi)
    Xo, _, _ = cholgs(Psi)
    _, _, theta, _ = rayleigh_ritz(H.apply, Xo)
    assert np.abs(theta - ref).max() < 1e-10


def test_rayleigh_ritz_courant_fischer_and_rotation():
    m, H = wells_system()
    lam = np.linalg.eigvalsh(H.dense())
    Xo, _, _ = cholgs(synth.random_block(5, m.ndofs, 8))
    X, W, theta, Hh = rayleigh_ritz(H.apply, Xo)
    assert np.all(np.diff(theta) >= 0)
    assert np.all(theta >= lam[:8] - 1e-12)
    assert np.abs(X.T @ X - np.eye(8)).max() < 1e-13
    assert np.abs(W - H.apply(X)).max() < 1e-11
    assert np.abs(X.T @ W - np.diag(theta)).max() < 1e-11
    # sign convention: largest-|.| entry of each column of Q = Xo^T X is positive
    Q = Xo.T @ X
    idx = np.argmax(np.abs(Q), axis=0)
    assert np.all(Q[idx, np.arange(8)] > 0)


def test_residuals_exact_and_bauer_fike():
    m, H = wells_system()
    lam, V = np.linalg.eigh(H.dense())
    W = H.apply(V[:, :5])
    r, rg = residuals(V[:, :5], W, lam[:5], m.mass)
    assert r.max() < 1e-11 and rg.max() < 1e-11
    Xo, _, _ = cholgs(synth.random_block(6, m.ndofs, 4))
    X, W, theta, _ = rayleigh_ritz(H.apply, Xo)
    r = residuals(X, W, theta)
    for i in range(4):
        assert r[i] >= np.min(np.abs(lam - theta[i])) - 1e-12
    # GHEP form ||H psi - theta M psi|| / ||psi|| with psi = M^-1/2 x, by direct formula
    _, rg = residuals(X, W, theta, m.mass)
    psi = X / np.sqrt(m.mass)[:, None]
    Hpsi = np.sqrt(m.mass)[:, None] * W          # H psi = M^1/2 H~ x
    Mpsi = m.mass[:, None] * psi
    ref = np.linalg.norm(Hpsi - Mpsi * theta[None, :], axis=0) / np.linalg.norm(psi, axis=0)
    assert np.allclose(rg, ref, rtol=1e-12)


def test_passes_converge_to_dense_eigenvalues():
    m, H = wells_system(ncell=2, p=3, nl=True)
    lam = np.linalg.eigvalsh(H.dense())
    N, B = 12, 6
    X = synth.random_block(7, m.ndofs, N)
    tmin, tmax, b = lanczos_bounds(H.apply, synth.counter_uniform(8, m.ndofs), 20)
    bd = first_pass_bounds(tmin, b, N, m.ndofs)
    for _ in range(25):
        X, W, theta, r, bd = chfsi_pass(H, X, B, 10, bd)
    assert np.abs(theta[:8] - lam[:8]).max() < 1e-9
    assert r[:8].max() < 1e-6
    assert np.all(theta >= lam[:N] - 1e-12)


def test_scaled_and_unscaled_filters_span_the_same_space():
    m, H = wells_system()
    X = synth.random_block(9, m.ndofs, 6)
    b1 = Bounds(a=4.0, b=110.0, a0=-1.5)
    b2 = Bounds(a=4.0, b=110.0)
    t1 = rayleigh_ritz(H.apply, cholgs(chebyshev_filter(H.apply, X, 8, b1))[0])[2]
    t2 = rayleigh_ritz(H.apply, cholgs(chebyshev_filter(H.apply, X, 8, b2))[0])[2]
    assert np.abs(t1 - t2).max() < 1e-10


def test_free_electron_passes_match_kronecker_sums():
    """V = 0 on a cube: converged Ritz values equal half-sums of three 1D spectra."""
    from test_oracle_hamiltonian import one_d_operator
    L, n, p = 8.0, 3, 3
    m = oracle.PeriodicMesh(L, n, p)
    H = oracle.Hamiltonian(m)
    mu = np.linalg.eigvalsh(one_d_operator(L, n, p)[2])
    sums = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel()) / 2
    N = 33
    X = synth.random_block(10, m.ndofs, N)
    tmin, tmax, b = lanczos_bounds(H.apply, synth.counter_uniform(12, m.ndofs), 20)
    bd = first_pass_bounds(tmin, b, N, m.ndofs)
    for _ in range(30):
        X, W, theta, r, bd = chfsi_pass(H, X, 11, 12, bd)
    assert np.abs(theta[:27] - sums[:27]).max() < 1e-10
