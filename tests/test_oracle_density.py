"""Oracle pins for spectrum splitting, the Fermi level and the density (Alg. 2, Alg. 3)."""
import numpy as np
import pytest

import oracle
import synth
from oracle.density import fermi_dirac, fermi_level, rayleigh_ritz_split, density, KB_HA_PER_K
from test_oracle_chfsi import wells_system

KT = 500.0 * KB_HA_PER_K          # the paper's smearing temperature, 500 K


def test_fermi_dirac_closed_form():
    assert abs(fermi_dirac(0.3, 0.3, KT) - 0.5) < 1e-15
    x = np.linspace(-0.01, 0.01, 7)
    f = fermi_dirac(x, 0.0, KT)
    assert np.allclose(f + fermi_dirac(-x, 0.0, KT), 1.0, atol=1e-15)    # particle-hole symmetry
    assert abs(fermi_dirac(KT * np.log(3.0), 0.0, KT) - 0.25) < 1e-14


def test_fermi_level_recovers_the_electron_count():
    eps = np.sort(np.random.default_rng(0).uniform(0.0, 0.05, 12))
    for ne in (2 * 20 + 0.5, 2 * 20 + 7.0, 2 * 20 + 23.5):
        mu = fermi_level(eps, 20, ne, KT)
        assert abs(2 * (20 + fermi_dirac(eps, mu, KT).sum()) - ne) < 1e-10
    # two levels kT apart holding one electron pair: mu sits halfway by f(-x) + f(x) = 1
    mu = fermi_level(np.array([0.15 - 0.5 * KT, 0.15 + 0.5 * KT]), 5, 2 * 5 + 2.0, KT)
    assert abs(mu - 0.15) < 1e-13
    with pytest.raises(ValueError):
        fermi_level(eps, 20, 2 * 20, KT)


def _converged_basis(m, H, N):
    lam, V = np.linalg.eigh(H.dense())
    X = V[:, :N] @ np.linalg.qr(synth.random_block(3, N, N))[0]   # rotated: same span, not Ritz vectors
    return lam, V, X


def test_split_ritz_pairs_are_the_top_of_the_full_set():
    m, H = wells_system(nl=True)
    N, nfr = 14, 5
    lam, V, X = _converged_basis(m, H, N)
    th_fr, Xfr, th = rayleigh_ritz_split(H.apply, X, nfr)
    assert np.abs(th - lam[:N]).max() < 1e-11
    assert np.abs(th_fr - lam[N - nfr:N]).max() < 1e-11
    assert np.abs(Xfr.T @ Xfr - np.eye(nfr)).max() < 1e-12
    assert np.abs(H.apply(Xfr) - Xfr * th_fr).max() < 1e-9


def test_density_split_formula_equals_occupied_sum():
    """Alg. 3's split formula equals 2 sum_i f_i |psi^_i|^2 with f = 1 below the window."""
    m, H = wells_system(nl=True)
    N, nfr = 14, 5
    lam, V, X = _converged_basis(m, H, N)
    th_fr, Xfr, th = rayleigh_ritz_split(H.apply, X, nfr)
    mu = fermi_level(th_fr, N - nfr, 2 * (N - nfr) + 4.3, KT)
    f = fermi_dirac(th_fr, mu, KT)
    rho = density(H, X, Xfr, f)
    occ = np.concatenate([np.ones(N - nfr), f])
    ref = np.zeros_like(rho)
    s = 1.0 / np.sqrt(m.mass)
    for c in range(m.ncells):
        P = H.Nq @ (s[m.cell_map[c], None] * V[m.cell_map[c], :N])
        ref[c] = 2.0 * (P * P) @ occ
    assert np.abs(rho - ref).max() < 1e-11 * np.abs(ref).max()
    assert rho.min() > -1e-12


def test_density_integrates_to_the_electron_count_with_gll_points():
    """With the GLL rule (quadrature points = nodes) int rho = 2 sum f_i psi^T M psi = N_e exactly."""
    m, H = wells_system(nl=False, vquad=1)
    N, nfr = 12, 4
    lam, V, X = _converged_basis(m, H, N)
    th_fr, Xfr, th = rayleigh_ritz_split(H.apply, X, nfr)
    ne = 2 * (N - nfr) + 3.1
    mu = fermi_level(th_fr, N - nfr, ne, KT)
    rho = density(H, X, Xfr, fermi_dirac(th_fr, mu, KT))
    total = np.sum(rho * (H.Wq * m.detJ)[None, :])
    assert abs(total - ne) < 1e-11
