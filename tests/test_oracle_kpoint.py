"""Oracle pins for the Bloch k-point Hamiltonian H~^k and the complex ChFSI steps (Sec. 2.1,
the reduced Kohn-Sham equation after Eq. bloch; Eq. chebyfilter, Alg. 2 with complex
blocks).  Independent routes: 1D operators assembled here and combined as a Kronecker sum,
the free-electron closed form 1/2 |k + G|^2, Bloch folding of a doubled supercell at the
Gamma point (which fixes the sign of the projector phases against the -i k.grad term),
dense eigensolves, and invariants."""
import math
import numpy as np
import pytest

import oracle
import synth
from oracle.basis import gll_rule, lagrange_deriv_table
from oracle.chfsi import Bounds, chebyshev_filter
from oracle import kpoint


def system(L, n, p, cent, hc, w=1.0, rc=2.5):
    m = oracle.PeriodicMesh(L, n, p)
    H = oracle.Hamiltonian(m)
    H.set_potential(synth.gaussian_wells(m.quad_xyz(0).reshape(-1, 3), cent, 2.0, 1.0, L))
    nl = None
    if hc is not None:
        rp, nd, chi = synth.projector_csr(m.node_xyz(), cent, w, rc, L)
        disp = synth.projector_disp(m.node_xyz(), cent, rc, L)
        H.set_nonlocal(hc, rp, nd, chi)
        nl = (hc, rp, nd, chi, disp)
    return m, H, nl


def bloch(H, k, nl):
    B = kpoint.BlochHamiltonian(H, k)
    if nl is not None:
        B.set_nonlocal(*nl)
    return B


def atoms(seed, n, L):
    s = synth.Stream(seed)
    cent = np.array([[L * s.uniform() for _ in range(3)] for _ in range(n)])
    hc = np.array([0.5 + 1.5 * s.uniform() for _ in range(4 * n)])
    return cent, hc


def one_d_bloch(L, n, p, k):
    """1D periodic operator 1/2 K~1 - i k G~1 + 1/2 k^2, assembled here from the 1D GLL
    stiffness int l_a' l_b' and derivative int l_a l_b' (both exact under GLL: degree 2p-2
    and 2p-1), Loewdin-scaled by the 1D lumped mass."""
    x, w = gll_rule(p)
    D = lagrange_deriv_table(x, x)           # D[i, b] = l_b'(x_i)
    h = L / n
    kloc = (2.0 / h) * (D.T * w) @ D
    gloc = w[:, None] * D                    # int l_a l_b' dx = w_a l_b'(x_a)
    g = n * p
    K1 = np.zeros((g, g))
    G1 = np.zeros((g, g))
    M1 = np.zeros(g)
    for c in range(n):
        idx = [(c * p + a) % g for a in range(p + 1)]
        K1[np.ix_(idx, idx)] += kloc
        G1[np.ix_(idx, idx)] += gloc
        M1[idx] += w * h / 2
    s = 1.0 / np.sqrt(M1)
    Kt = s[:, None] * K1 * s[None, :]
    Gt = s[:, None] * G1 * s[None, :]
    return 0.5 * Kt - 1j * k * Gt + 0.5 * k * k * np.eye(g)


def test_k_zero_is_the_gamma_operator():
    cent, hc = atoms(1, 2, 6.0)
    m, H, nl = system(6.0, 2, 3, cent, hc)
    B = bloch(H, (0.0, 0.0, 0.0), nl)
    X = synth.random_block(4, m.ndofs, 6).view(np.complex128)
    Y = B.apply(X)
    ref = H.apply(X.real) + 1j * H.apply(X.imag)
    assert np.abs(Y - ref).max() < 1e-13 * np.abs(ref).max()


def test_hermitian_with_projectors():
    cent, hc = atoms(2, 2, 6.0)
    m, H, nl = system(6.0, (2, 3, 2), 3, cent, hc)
    D = bloch(H, (0.31, -0.2, 0.45), nl).dense()
    assert np.abs(D - D.conj().T).max() < 1e-13 * np.abs(D).max()
    assert np.abs(D.imag).max() > 0.05          # the k terms are there
    # the nonlocal part is PSD: adding it raises every eigenvalue (Weyl)
    Dl = bloch(H, (0.31, -0.2, 0.45), None).dense()
    assert np.all(np.linalg.eigvalsh(D) >= np.linalg.eigvalsh(Dl) - 1e-10)


@pytest.mark.parametrize("p,n,L,k", [(2, (2, 3, 2), (4.0, 5.0, 6.0), (0.3, -0.7, 0.2)),
                                     (4, (3, 2, 2), (6.0, 6.5, 7.0), (0.5, 0.1, -0.35)),
                                     (1, (3, 2, 4), (3.0, 4.0, 5.0), (0.9, -0.2, 0.4)),
                                     (8, (2, 2, 2), (5.0, 5.5, 6.0), (-0.3, 0.6, 0.15))])
def test_free_electron_is_kronecker_sum_of_1d_bloch_operators(p, n, L, k):
    """V = 0: H~^k = A_z (x) I (x) I + I (x) A_y (x) I + I (x) I (x) A_x (x fastest), each A_d the
    1D operator above; a transposed component, a wrong sign of i or a missing 1/2|k|^2 fails."""
    m = oracle.PeriodicMesh(L, n, p)
    H = oracle.Hamiltonian(m)
    B = kpoint.BlochHamiltonian(H, k)
    A = [one_d_bloch(L[d], n[d], p, k[d]) for d in range(3)]
    I = [np.eye(m.g[d]) for d in range(3)]
    ref = (np.kron(I[2], np.kron(I[1], A[0])) + np.kron(I[2], np.kron(A[1], I[0]))
           + np.kron(A[2], np.kron(I[1], I[0])))
    Bd = B.dense()
    assert np.abs(Bd - ref).max() < 1e-12 * np.abs(ref).max()
    X = synth.random_block(3, m.ndofs, 8).view(np.complex128)
    assert np.abs(B.apply(X) - ref @ X).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("k", [0.0, 0.37, -1.1])
def test_1d_bloch_operator_converges_to_free_electron(k):
    """Spectrum of the 1D operator -> 1/2 (k + 2 pi n / L)^2 (spectral accuracy at p = 8)."""
    L = 6.0
    lam = np.linalg.eigvalsh(one_d_bloch(L, 12, 8, k))[:9]
    G = 2 * math.pi / L * np.arange(-6, 7)
    ref = np.sort(0.5 * (k + G) ** 2)[:9]
    assert np.abs(lam - ref).max() < 1e-9


def test_3d_free_electron_levels():
    """The lowest levels of H~^k on a p = 4 mesh against 1/2 |k + G|^2."""
    L = 5.0
    k = np.array([0.2, -0.35, 0.1])
    m = oracle.PeriodicMesh(L, 3, 4)
    B = kpoint.BlochHamiltonian(oracle.Hamiltonian(m), k)
    lam = np.linalg.eigvalsh(B.dense())[:10]
    n = np.arange(-2, 3)
    G = 2 * math.pi / L * np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3)
    ref = np.sort(0.5 * np.sum((k + G) ** 2, axis=1))[:10]
    assert np.abs(lam - ref).max() < 2e-4 * ref.max()


def _folding_gap(flip=False):
    L = 6.0
    cent, hc = atoms(5, 2, L)
    m, H, nl = system((L, L, L), (3, 3, 3), 4, cent, hc)
    ev = []
    for kx in (0.0, math.pi / L):
        hc_, rp, nd, chi, disp = nl
        B = bloch(H, (kx, 0.0, 0.0), (hc_, rp, nd, chi, -disp if flip else disp))
        ev.append(np.linalg.eigvalsh(B.dense())[:12])
    cent2 = np.concatenate([cent, cent + np.array([L, 0.0, 0.0])])
    _, H2, _ = system((2 * L, L, L), (6, 3, 3), 4, cent2, np.concatenate([hc, hc]))
    es = np.linalg.eigvalsh(H2.dense())[:12]
    return np.abs(np.sort(np.concatenate(ev))[:12] - es).max()


def test_bloch_folding_matches_doubled_supercell():
    """The Gamma spectrum of the cell doubled along x (same mesh, atoms repeated) is the union
    of the cell's spectra at k = 0 and k = pi/L x: both discretisations converge to it
    (2e-4 Ha at p = 4, 2e-5 at p = 5, 1.4e-6 at p = 6 on this system).  Projector phases of
    the wrong sign against the -i k.grad term miss it by 0.11 Ha."""
    assert _folding_gap() < 1e-3


def test_folding_pin_catches_a_flipped_phase():
    assert _folding_gap(flip=True) > 0.05


@pytest.mark.parametrize("scaled", [False, True])
def test_complex_filter_scalar_identity_on_eigenvectors(scaled):
    cent, hc = atoms(3, 2, 6.0)
    m, H, nl = system(6.0, 2, 3, cent, hc)
    B = bloch(H, (0.4, 0.1, -0.2), nl)
    lam, V = np.linalg.eigh(B.dense())
    bd = Bounds(a=lam[10], b=lam[-1] + 0.5, a0=lam[0] - 0.1 if scaled else math.nan)
    deg = 9
    e, c = (bd.b - bd.a) / 2, (bd.b + bd.a) / 2
    x = (lam - c) / e
    t = np.where(np.abs(x) <= 1, np.cos(deg * np.arccos(np.clip(x, -1, 1))),
                 np.sign(x) ** deg * np.cosh(deg * np.arccosh(np.maximum(np.abs(x), 1))))
    if scaled:
        x0 = (bd.a0 - c) / e
        t = t / (np.sign(x0) ** deg * np.cosh(deg * np.arccosh(abs(x0))))
    cols = [0, 3, 10, 50, len(lam) - 1]
    Y = chebyshev_filter(B.apply, V[:, cols], deg, bd)
    assert Y.dtype == np.complex128
    assert np.abs(Y - V[:, cols] * t[cols][None, :]).max() < 1e-11 * max(1.0, np.abs(t).max())


def test_complex_cholgs_orthonormal_and_span():
    X = synth.random_block(7, 300, 16).view(np.complex128)
    Xo, S, L = kpoint.cholgs(X)
    assert np.abs(Xo.conj().T @ Xo - np.eye(8)).max() < 1e-13
    assert np.allclose(L @ L.conj().T, S, atol=1e-12)
    P0 = X @ np.linalg.solve(X.conj().T @ X, X.conj().T)
    assert np.abs(Xo @ Xo.conj().T - P0).max() < 1e-12


def test_complex_rr_courant_fischer_phase_and_residuals():
    cent, hc = atoms(4, 2, 6.0)
    m, H, nl = system(6.0, 2, 3, cent, hc)
    B = bloch(H, (0.2, 0.3, 0.0), nl)
    lam = np.linalg.eigvalsh(B.dense())
    X, _, _ = kpoint.cholgs(synth.random_block(2, m.ndofs, 20).view(np.complex128))
    Xr, W, theta, Hh = kpoint.rayleigh_ritz(B.apply, X)
    assert np.all(np.diff(theta) >= 0)
    assert np.all(theta >= lam[:10] - 1e-10)                # Courant-Fischer
    assert np.abs(Hh - Hh.conj().T).max() == 0.0
    Q = X.conj().T @ Xr                                       # the phases are fixed on Q
    piv = Q[np.argmax(np.abs(Q), axis=0), np.arange(10)]
    assert np.all(np.abs(piv.imag) < 1e-12) and np.all(piv.real > 0)
    r = kpoint.residuals(Xr, W, theta)
    assert np.allclose(r, np.linalg.norm(B.apply(Xr) - Xr * theta, axis=0), rtol=1e-10)
    assert np.all(r >= np.min(np.abs(theta[:, None] - lam[None, :]), axis=1) - 1e-10)   # Bauer-Fike


def test_lanczos_on_the_real_form_brackets_the_spectrum():
    cent, hc = atoms(6, 2, 6.0)
    m, H, nl = system(6.0, 2, 3, cent, hc)
    B = bloch(H, (0.5, -0.1, 0.25), nl)
    lam = np.linalg.eigvalsh(B.dense())
    tmin, tmax, b = kpoint.spectrum_bounds(B, synth.counter_uniform(3, 2 * m.ndofs), 20)
    assert b >= lam[-1] - 1e-9
    assert lam[0] - 1e-9 <= tmin and tmax <= lam[-1] + 1e-9


def test_complex_passes_converge_to_dense_eigenvalues():
    cent, hc = atoms(8, 2, 6.0)
    m, H, nl = system(6.0, 2, 3, cent, hc)
    B = bloch(H, (0.3, 0.2, -0.15), nl)
    lam = np.linalg.eigvalsh(B.dense())
    X = synth.random_block(11, m.ndofs, 2 * 12).view(np.complex128)
    tmin, _, b = kpoint.spectrum_bounds(B, synth.counter_uniform(3, 2 * m.ndofs), 20)
    bd = oracle.first_pass_bounds(tmin, b, 12, m.ndofs)
    for _ in range(12):
        X, W, theta, r, bd = kpoint.chfsi_pass(B, X, 6, 12, bd)
    ok = r < 1e-7
    assert ok[:8].all()
    assert np.abs(theta[ok] - lam[:12][ok]).max() < 1e-9


def test_complex_generalised_residual_reduces_to_the_real_one():
    """At a real block the complex residuals (both forms) are the real oracle's; on exact
    eigenvectors of H~^k both vanish."""
    cent, hc = atoms(9, 2, 6.0)
    m, H, nl = system(6.0, 2, 3, cent, hc)
    X = synth.random_block(3, m.ndofs, 5)
    W = H.apply(X)
    th = np.linspace(-1.0, 1.0, 5)
    r0, g0 = oracle.residuals(X, W, th, m.mass)
    r1, g1 = kpoint.residuals(X.astype(np.complex128), W.astype(np.complex128), th, m.mass)
    assert np.allclose(r0, r1, rtol=1e-14) and np.allclose(g0, g1, rtol=1e-14)
    B = bloch(H, (0.2, 0.1, -0.3), nl)
    lam, V = np.linalg.eigh(B.dense())
    r, g = kpoint.residuals(V[:, :4], B.apply(V[:, :4]), lam[:4], m.mass)
    assert r.max() < 1e-11 and g.max() < 1e-11


def test_realification_identities_used_by_the_complex_cholgs_and_rr():
    """The library runs complex CholGS / Rayleigh-Ritz on real views (M x 2N, real and imaginary
    parts interleaved).  Checked here in numpy: the complex Gram is read off the real Gram
    G = Xr^T Xr; the interleaved real form rho(S) of S = X^H X has the real Cholesky factor
    rho(L) (L the complex one); the real solve with rho(L) gives the real view of X L^-H; and
    right multiplication by rho(Q) gives the real view of X Q."""
    X = synth.random_block(3, 200, 2 * 7).view(np.complex128)
    N = X.shape[1]
    Xr = X.view(np.float64)
    G = Xr.T @ Xr

    def rho(A):
        R = np.zeros((2 * A.shape[0], 2 * A.shape[1]))
        R[0::2, 0::2] = A.real
        R[1::2, 1::2] = A.real
        R[0::2, 1::2] = A.imag
        R[1::2, 0::2] = -A.imag
        return R
    S = X.conj().T @ X
    Sg = (G[0::2, 0::2] + G[1::2, 1::2]) + 1j * (G[0::2, 1::2] - G[1::2, 0::2])
    assert np.allclose(Sg, S, atol=1e-12)
    L = np.linalg.cholesky(S)
    Lr = np.linalg.cholesky(rho(S))
    assert np.allclose(Lr, rho(L), atol=1e-12)
    Xo, _, _ = kpoint.cholgs(X)
    Xo_real = Xr @ np.linalg.inv(Lr).T
    assert np.allclose(Xo_real, np.ascontiguousarray(Xo).view(np.float64), atol=1e-12)
    Q = np.linalg.qr(synth.random_block(4, N, 2 * N).view(np.complex128))[0]
    assert np.allclose(Xr @ rho(Q), np.ascontiguousarray(X @ Q).view(np.float64), atol=1e-12)
    assert np.allclose(rho(Q.conj().T), rho(Q).T) and np.allclose(rho(L @ Q), rho(L) @ rho(Q))
