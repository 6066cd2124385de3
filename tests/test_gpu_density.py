"""Spectrum splitting, Fermi level and density (Alg. 2 step 3a, Alg. 3) through the C ABI
against the FP64 oracle on the same inputs, plus a sampled-cell check at full size."""
import numpy as np
import pytest

import oracle
import synth
from oracle.density import fermi_dirac, fermi_level, rayleigh_ritz_split, density, KB_HA_PER_K
from systems import oracle_system, gpu_system, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KT = 500.0 * KB_HA_PER_K


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


CASES = {
    "p4_432_nl_gauss": small_case(0, n=(4, 3, 2), p=4, L=8.0, nl=True),
    "p3_333_gll": small_case(2, n=(3, 3, 3), p=3, L=6.0, nl=False, vquad=1),
    "p6_223_nl_gauss": small_case(1, n=(2, 2, 3), p=6, L=7.0, nl=True),
}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request, dg):
    c = CASES[request.param]
    om, oh = oracle_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    lam, V = np.linalg.eigh(oh.dense())
    yield om, oh, mesh, ham, lam, V
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)


def _basis(V, N, seed=3):
    return V[:, :N] @ np.linalg.qr(synth.random_block(seed, N, N))[0]


@pytest.mark.parametrize("prec", [0, 2])
def test_split_rayleigh_ritz(dg, pair, prec):
    om, oh, mesh, ham, lam, V = pair
    N, nfr = 16, 6
    X0 = _basis(V, N)
    th_fr, Xfr_o, th = rayleigh_ritz_split(oh.apply, X0, nfr)
    X = torch.from_numpy(X0).cuda()
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    Xfr = torch.empty((om.ndofs, nfr), dtype=torch.float64, device="cuda")
    dg.dftfe_rayleigh_ritz_split(ham, X, nfr, ev, Xfr, prec)
    tol = 1e-11 if prec == 0 else 1e-6
    assert np.abs(ev.cpu().numpy() - th).max() < tol
    assert np.array_equal(X.cpu().numpy(), X0)                      # input untouched
    gaps = np.minimum(np.r_[np.inf, np.diff(th_fr)], np.r_[np.diff(th_fr), np.inf])
    ok = gaps > 1e-4
    xf = Xfr.cpu().numpy()
    assert np.abs(xf[:, ok] - Xfr_o[:, ok]).max() < (1e-8 if prec == 0 else 1e-4)


def test_fermi_level(dg, pair):
    om, oh, mesh, ham, lam, V = pair
    eps = lam[10:16]
    for ne in (2 * 10 + 0.7, 2 * 10 + 5.5, 2 * 10 + 11.3):
        mu_o = fermi_level(eps, 10, ne, KT)
        f = torch.empty(6, dtype=torch.float64, device="cuda")
        mu = dg.dftfe_fermi_level(torch.from_numpy(eps).cuda(), 10, ne, KT, f)
        assert abs(mu - mu_o) < 1e-12
        assert np.abs(f.cpu().numpy() - fermi_dirac(eps, mu_o, KT)).max() < 1e-12
    with pytest.raises(dg.DftfeError):
        dg.dftfe_fermi_level(torch.from_numpy(eps).cuda(), 10, 2 * 10 + 12.0, KT, f)


def test_density_matches_oracle(dg, pair):
    om, oh, mesh, ham, lam, V = pair
    N, nfr = 16, 6
    X0 = _basis(V, N)
    th_fr, Xfr0, th = rayleigh_ritz_split(oh.apply, X0, nfr)
    ne = 2 * (N - nfr) + 4.2
    f0 = fermi_dirac(th_fr, fermi_level(th_fr, N - nfr, ne, KT), KT)
    ref = density(oh, X0, Xfr0, f0)
    rho = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    dg.dftfe_density(ham, torch.from_numpy(X0).cuda(), torch.from_numpy(Xfr0).cuda(),
                     torch.from_numpy(f0).cuda(), rho)
    got = rho.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    if CASES_KEY(pair) == "gll":
        assert abs(np.sum(got * (oh.Wq * om.detJ)[None, :]) - ne) < 1e-10


def CASES_KEY(pair):
    om, oh = pair[0], pair[1]
    return "gll" if oh.vquad == 1 else "gauss"


def test_density_without_split_states(dg, pair):
    om, oh, mesh, ham, lam, V = pair
    X0 = _basis(V, 8)
    ref = density(oh, X0, np.zeros((om.ndofs, 0)), np.zeros(0))
    rho = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    dg.dftfe_density(ham, torch.from_numpy(X0).cuda(), None, None, rho)
    assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_density_full_size_sampled_cells(dg):
    """2,985,984 DoFs, p = 6: density of 32 + 8 seeded columns on sampled cells."""
    wl = synth.lattice_atoms(0)
    mesh = dg.dftfe_mesh_create(wl.L, wl.ncell, wl.degree)
    ham = dg.dftfe_ham_create(mesh)
    _, qxyz = dg.dftfe_mesh_coords(mesh, nodes=False)
    v = synth.gaussian_wells(qxyz.reshape(-1, 3), wl.centres, wl.depth, wl.width, wl.L)
    dg.dftfe_ham_set_potential(ham, torch.from_numpy(v).cuda())
    om = oracle.PeriodicMesh(wl.L, wl.ncell, wl.degree)
    oh = oracle.Hamiltonian(om)
    M, N, nfr = om.ndofs, 32, 8
    Xo = torch.empty((M, N), dtype=torch.float64, device="cuda")
    Xf = torch.empty((M, nfr), dtype=torch.float64, device="cuda")
    dg.dftfe_random_uniform(Xo, 21)
    dg.dftfe_random_uniform(Xf, 22)
    f = np.linspace(0.1, 0.9, nfr)
    rho = torch.empty((om.ncells, oh.nq), dtype=torch.float64, device="cuda")
    dg.dftfe_density(ham, Xo, Xf, torch.from_numpy(f).cuda(), rho)
    cells = np.array([0, 1, 577, 6000, om.ncells - 1])
    ref = density(oh, synth.random_block(21, M, N), synth.random_block(22, M, nfr), f, cells=cells)
    got = rho[torch.from_numpy(cells).cuda()].cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)
