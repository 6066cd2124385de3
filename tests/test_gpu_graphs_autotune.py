"""CUDA graphs of the pass's filter phase and the FP64 cell-kernel autotuner: both change only
how the work is launched, so every result must be bit-identical to the plain launches, and
graphed and autotuned passes must match the FP64 oracle."""
import math
import numpy as np
import pytest

import oracle
import synth
from systems import gpu_system, oracle_system, small_case

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


def _sys(dg, c):
    return gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])


def _disp(dg, mesh, c):
    nxyz, _ = dg.dftfe_mesh_coords(mesh, quad=False)
    cent, w, rc, hc = c["proj"]
    return synth.projector_disp(nxyz, cent, rc, c["L"])


@pytest.mark.parametrize("prec_name", ["DFTFE_FP64", "DFTFE_MIXED_TF32X3"])
@pytest.mark.parametrize("scaled", [True, False])
def test_graphed_pass_is_bit_identical(dg, prec_name, scaled):
    prec = getattr(dg, prec_name)
    c = small_case(0, n=(4, 3, 2), p=4, L=8.0, nl=True)
    (m1, h1), (m2, h2) = _sys(dg, c), _sys(dg, c)
    dg.dftfe_ham_use_graphs(h2, True)
    M = dg.dftfe_mesh_info(m1)[0]
    N, blk, deg = 20, 8, 9
    X0 = torch.from_numpy(synth.random_block(5, M, N)).cuda()
    X1, X2 = X0.clone(), X0.clone()
    b = dg.dftfe_spectrum_bounds(h1, 20, 3, N)
    if not scaled:
        b.a0 = math.nan
    b1, b2 = dg.make_bounds(b.a, b.b, b.a0), dg.make_bounds(b.a, b.b, b.a0)
    e1, r1, e2, r2 = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4))
    for it in range(4):
        dg.dftfe_chfsi_pass(h1, X1, blk, deg, b1, e1, r1, prec)
        dg.dftfe_chfsi_pass(h2, X2, blk, deg, b2, e2, r2, prec)
        assert torch.equal(e1, e2) and torch.equal(r1, r2) and torch.equal(X1, X2), it
        assert (b1.a, b1.a0) == (b2.a, b2.a0) or (math.isnan(b1.a0) and b1.a == b2.a)
    replays, inst = dg.dftfe_graph_query(h2)
    assert replays == 3 and inst >= 1                  # the first pass ran without a graph
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_destroy(h)
        dg.dftfe_mesh_destroy(m)


def test_graphed_pass_survives_a_new_potential(dg):
    """A new potential adds the split-tile launches to the next mixed filter (another graph
    topology): the executable is instantiated afresh and the results stay identical."""
    c = small_case(1, n=(2, 2, 3), p=6, L=7.0, nl=True)
    (m1, h1), (m2, h2) = _sys(dg, c), _sys(dg, c)
    dg.dftfe_ham_use_graphs(h2, True)
    M = dg.dftfe_mesh_info(m1)[0]
    _, qxyz = dg.dftfe_mesh_coords(m1, nodes=False)
    N, blk, deg = 12, 12, 6
    X1 = torch.from_numpy(synth.random_block(6, M, N)).cuda()
    X2 = X1.clone()
    b = dg.dftfe_spectrum_bounds(h1, 20, 3, N)
    b1, b2 = dg.make_bounds(b.a, b.b, b.a0), dg.make_bounds(b.a, b.b, b.a0)
    e1, r1, e2, r2 = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4))
    for it in range(4):
        if it == 2:
            v = synth.gaussian_wells(qxyz.reshape(-1, 3), c["centres"] + 0.05, c["depth"], c["width"], c["L"])
            for h in (h1, h2):
                dg.dftfe_ham_set_potential(h, torch.from_numpy(v).cuda())
        dg.dftfe_chfsi_pass(h1, X1, blk, deg, b1, e1, r1, dg.DFTFE_MIXED_TF32X3)
        dg.dftfe_chfsi_pass(h2, X2, blk, deg, b2, e2, r2, dg.DFTFE_MIXED_TF32X3)
        assert torch.equal(e1, e2) and torch.equal(X1, X2), it
    replays, inst = dg.dftfe_graph_query(h2)
    assert replays == 3 and inst >= 2
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_destroy(h)
        dg.dftfe_mesh_destroy(m)


@pytest.mark.parametrize("prec_name", ["DFTFE_FP64", "DFTFE_MIXED_TF32X3"])
def test_graphed_complex_pass_is_bit_identical(dg, prec_name):
    prec = getattr(dg, prec_name)
    c = small_case(0, n=(4, 3, 2), p=4, L=8.0, nl=True)
    (m1, h1), (m2, h2) = _sys(dg, c), _sys(dg, c)
    k = (0.3, -0.2, 0.45)
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_set_kpoint(h, k, _disp(dg, m, c))
    dg.dftfe_ham_use_graphs(h2, True)
    M = dg.dftfe_mesh_info(m1)[0]
    N, blk, deg = 10, 4, 7
    X1 = torch.from_numpy(synth.random_block(8, M, 2 * N).view(np.complex128)).cuda()
    X2 = X1.clone()
    b = dg.dftfe_spectrum_bounds_z(h1, 20, 3, N)
    b1, b2 = dg.make_bounds(b.a, b.b, b.a0), dg.make_bounds(b.a, b.b, b.a0)
    e1, r1, e2, r2 = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4))
    for it in range(3):
        dg.dftfe_chfsi_pass_z(h1, X1, blk, deg, b1, e1, r1, prec)
        dg.dftfe_chfsi_pass_z(h2, X2, blk, deg, b2, e2, r2, prec)
        assert torch.equal(e1, e2) and torch.equal(X1, X2), it
    assert dg.dftfe_graph_query(h2)[0] == 2
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_destroy(h)
        dg.dftfe_mesh_destroy(m)


@pytest.mark.parametrize("case", [small_case(0, n=(4, 3, 2), p=4, L=8.0, nl=True),
                                  small_case(1, n=(2, 2, 3), p=6, L=7.0, nl=True)])
def test_autotuned_apply_is_bit_identical(dg, case):
    (m1, h1), (m2, h2) = _sys(dg, case), _sys(dg, case)
    dg.dftfe_ham_autotune(h2, True)
    M, _, nc, _ = dg.dftfe_mesh_info(m1)
    assert dg.dftfe_autotune_query(h2, 40)[0] == -1
    X = torch.from_numpy(synth.random_block(9, M, 40)).cuda()
    Y1, Y2 = torch.empty_like(X), torch.empty_like(X)
    dg.dftfe_ham_apply(h1, X, Y1)
    dg.dftfe_ham_apply(h2, X, Y2)
    assert torch.equal(Y1, Y2)
    rows, best, heur = dg.dftfe_autotune_query(h2, 40)
    assert rows == 0 or (rows % 64 == 0 and 64 <= rows <= (nc + 63) // 64 * 64)
    assert 0 < best <= heur
    dg.dftfe_ham_apply(h2, X, Y2)                      # tuned shape reused
    assert torch.equal(Y1, Y2)
    dg.dftfe_ham_autotune(h2, False)
    assert dg.dftfe_autotune_query(h2, 40)[0] == -1
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_destroy(h)
        dg.dftfe_mesh_destroy(m)


def test_autotuned_graphed_complex_pass_matches_plain(dg):
    c = small_case(1, n=(2, 2, 3), p=6, L=7.0, nl=True)
    (m1, h1), (m2, h2) = _sys(dg, c), _sys(dg, c)
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_set_kpoint(h, (math.pi / 7.0, 0.0, 0.1), _disp(dg, m, c))
    dg.dftfe_ham_autotune(h2, True)
    dg.dftfe_ham_use_graphs(h2, True)
    M = dg.dftfe_mesh_info(m1)[0]
    N = 16
    X1 = torch.from_numpy(synth.random_block(10, M, 2 * N).view(np.complex128)).cuda()
    X2 = X1.clone()
    b = dg.dftfe_spectrum_bounds_z(h1, 20, 4, N)
    b1, b2 = dg.make_bounds(b.a, b.b, b.a0), dg.make_bounds(b.a, b.b, b.a0)
    e1, r1, e2, r2 = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4))
    for _ in range(3):
        dg.dftfe_chfsi_pass_z(h1, X1, 8, 8, b1, e1, r1)
        dg.dftfe_chfsi_pass_z(h2, X2, 8, 8, b2, e2, r2)
        assert torch.equal(e1, e2) and torch.equal(X1, X2)
    assert dg.dftfe_autotune_query(h2, 16)[0] >= 0     # 8 complex columns = 16 real ones
    for h, m in ((h1, m1), (h2, m2)):
        dg.dftfe_ham_destroy(h)
        dg.dftfe_mesh_destroy(m)


@pytest.mark.parametrize("mode", ["graphed", "autotuned", "graphed+autotuned"])
def test_graphed_and_autotuned_passes_match_the_oracle(dg, mode):
    """Three passes with the graphed filter phase and/or the autotuned FP64 cell kernel against
    three passes of the FP64 oracle from the same seeded start and the oracle's own bounds:
    Ritz values within 1e-9 Ha, bounds updates within 1e-9 Ha."""
    c = small_case(0, n=(4, 3, 2), p=4, L=8.0, nl=True)
    om, oh = oracle_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    mesh, ham = _sys(dg, c)
    try:
        dg.dftfe_ham_use_graphs(ham, "graphed" in mode)
        dg.dftfe_ham_autotune(ham, "autotuned" in mode)
        N, blk, deg = 20, 8, 9
        X0 = synth.random_block(15, om.ndofs, N)
        tmin, _, b = oracle.lanczos_bounds(oh.apply, synth.counter_uniform(16, om.ndofs), 20)
        bo = oracle.first_pass_bounds(tmin, b, N, om.ndofs)
        bg = dg.make_bounds(bo.a, bo.b, bo.a0)
        X = torch.from_numpy(X0).cuda()
        ev = torch.empty(N, dtype=torch.float64, device="cuda")
        rs = torch.empty_like(ev)
        Xo = X0
        for it in range(3):
            dg.dftfe_chfsi_pass(ham, X, blk, deg, bg, ev, rs)
            Xo, _, theta, r, bo = oracle.chfsi_pass(oh, Xo, blk, deg, bo)
            assert np.abs(ev.cpu().numpy() - theta).max() < 1e-9, it
            assert abs(bg.a - bo.a) < 1e-9 and abs(bg.a0 - bo.a0) < 1e-9, it
        if "graphed" in mode:
            assert dg.dftfe_graph_query(ham)[0] == 2           # passes 2 and 3 replayed the graph
        if "autotuned" in mode:
            rows, best, heur = dg.dftfe_autotune_query(ham, blk)
            assert best > 0.0
    finally:
        dg.dftfe_ham_destroy(ham)
        dg.dftfe_mesh_destroy(mesh)
