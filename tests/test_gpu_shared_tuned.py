"""Hams that share one local operator (the k-points of one system), the split-precision
cell-kernel autotuner and the batch's shared tail workspace: every form gives the bits of
the plain form, and the shared operator follows its owner's potential."""
import numpy as np
import pytest

import synth
from systems import gpu_system, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KPTS = [(0.2, -0.1, 0.3), (0.0, 0.5, -0.25), (-0.3, 0.1, 0.0)]


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


def _case(seed=3, n=(4, 3, 2), p=5, L=8.0):
    return small_case(seed, n=n, p=p, L=L, nl=True)


def _kham(dg, c, mesh, ham, k):
    nxyz, _ = dg.dftfe_mesh_coords(mesh, quad=False)
    cent, w, rc, hc = c["proj"]
    rowptr, node, chi = synth.projector_csr(nxyz, cent, w, rc, c["L"])
    dg.dftfe_ham_set_nonlocal(ham, hc, rowptr, node, chi)
    dg.dftfe_ham_set_kpoint(ham, k, synth.projector_disp(nxyz, cent, rc, c["L"]))


def _start(dg, M, N, seed):
    Xr = torch.empty((M, 2 * N), dtype=torch.float64, device="cuda")
    dg.dftfe_random_uniform(Xr, seed)
    return Xr.view(torch.complex128)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_shared_kpoint_hams_match_independent_hams(dg, prec):
    """k-point hams made by dftfe_ham_create_shared from one Gamma-point ham give, pass for
    pass, the bits of k-point hams that each set the same potential themselves."""
    c = _case()
    P = dg.DFTFE_FP64 if prec == "fp64" else dg.DFTFE_MIXED_TF32X3
    mesh, src = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    shared = [dg.dftfe_ham_create_shared(src) for _ in KPTS]
    own = [gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], None) for _ in KPTS]
    try:
        for k, hs, (m2, ho) in zip(KPTS, shared, own):
            _kham(dg, c, mesh, hs, k)
            _kham(dg, c, m2, ho, k)
        M = dg.dftfe_mesh_info(mesh)[0]
        N, blk, deg = 12, 6, 8
        for i, (hs, (m2, ho)) in enumerate(zip(shared, own)):
            X1 = _start(dg, M, N, 40 + i)
            X2 = X1.clone()
            b1 = dg.dftfe_spectrum_bounds_z(hs, 20, 9, N)
            b2 = dg.dftfe_spectrum_bounds_z(ho, 20, 9, N)
            assert (b1.a, b1.b, b1.a0) == (b2.a, b2.b, b2.a0)
            e1 = torch.empty(N, dtype=torch.float64, device="cuda")
            r1, e2, r2 = torch.empty_like(e1), torch.empty_like(e1), torch.empty_like(e1)
            for _ in range(2):
                dg.dftfe_chfsi_pass_z(hs, X1, blk, deg, b1, e1, r1, P)
                dg.dftfe_chfsi_pass_z(ho, X2, blk, deg, b2, e2, r2, P)
            torch.cuda.synchronize()
            assert torch.equal(X1, X2) and torch.equal(e1, e2) and torch.equal(r1, r2), i
    finally:
        for h in shared:
            dg.dftfe_ham_destroy(h)
        dg.dftfe_ham_destroy(src)
        dg.dftfe_mesh_destroy(mesh)
        for m2, ho in own:
            dg.dftfe_ham_destroy(ho)
            dg.dftfe_mesh_destroy(m2)


def test_shared_operator_rules_and_new_potential(dg):
    """set_potential on a sharing ham and destroying the owner first are refused; a new
    potential on the owner reaches the sharing ham (its H~X equals that of an independent ham
    with the new potential, in FP64 and in the split precision)."""
    c = _case(seed=5, n=(3, 3, 2), p=4, L=7.0)
    mesh, src = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], None)
    hs = dg.dftfe_ham_create_shared(src)
    m2, ho = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], None)
    try:
        _, qxyz = dg.dftfe_mesh_coords(mesh)
        v2 = torch.from_numpy(synth.gaussian_wells(qxyz.reshape(-1, 3), c["centres"][:1], 3.0, 0.7, c["L"])).cuda()
        with pytest.raises(dg.DftfeError) as e:
            dg.dftfe_ham_set_potential(hs, v2)
        assert e.value.code == dg.DFTFE_ERR_STATE
        with pytest.raises(dg.DftfeError) as e:
            dg.dftfe_ham_destroy(src)
        assert e.value.code == dg.DFTFE_ERR_STATE
        with pytest.raises(dg.DftfeError) as e:
            dg.dftfe_ham_create_shared(hs)                  # a sharing ham owns no operator
        assert e.value.code == dg.DFTFE_ERR_ARG
        M = dg.dftfe_mesh_info(mesh)[0]
        X = torch.empty((M, 40), dtype=torch.float64, device="cuda")
        dg.dftfe_random_uniform(X, 3)
        for prec in (dg.DFTFE_FP64, dg.DFTFE_MIXED_TF32X3):
            Y1, Y2 = torch.empty_like(X), torch.empty_like(X)
            dg.dftfe_ham_apply(hs, X, Y1, prec)            # builds the owner's split plane
            dg.dftfe_ham_apply(ho, X, Y2, prec)
            torch.cuda.synchronize()
            assert torch.equal(Y1, Y2)
        dg.dftfe_ham_set_potential(src, v2)
        dg.dftfe_ham_set_potential(ho, v2)
        for prec in (dg.DFTFE_FP64, dg.DFTFE_MIXED_TF32X3, dg.DFTFE_FP64_SLICES):
            Y1, Y2 = torch.empty_like(X), torch.empty_like(X)
            dg.dftfe_ham_apply(hs, X, Y1, prec)
            dg.dftfe_ham_apply(ho, X, Y2, prec)
            torch.cuda.synchronize()
            assert torch.equal(Y1, Y2), prec
    finally:
        dg.dftfe_ham_destroy(hs)
        dg.dftfe_ham_destroy(src)
        dg.dftfe_mesh_destroy(mesh)
        dg.dftfe_ham_destroy(ho)
        dg.dftfe_mesh_destroy(m2)


def test_tuned_tf32x3_passes_are_bit_identical(dg):
    """With the autotuner on, the first split-precision cell launch times every shape of the
    kernel and keeps the fastest; the passes give the bits of untuned passes."""
    c = small_case(1, n=(4, 4, 3), p=6, L=9.0, nl=True)
    made = [gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
            for _ in range(2)]
    try:
        dg.dftfe_ham_autotune(made[1][1], True)
        assert dg.dftfe_autotune_query_mixed(made[1][1])[0] == -1
        M = dg.dftfe_mesh_info(made[0][0])[0]
        N = 40
        X1 = torch.empty((M, N), dtype=torch.float64, device="cuda")
        dg.dftfe_random_uniform(X1, 21)
        X2 = X1.clone()
        b1 = dg.dftfe_spectrum_bounds(made[0][1], 20, 5, N)
        b2 = dg.make_bounds(b1.a, b1.b, b1.a0)
        e1 = torch.empty(N, dtype=torch.float64, device="cuda")
        r1, e2, r2 = torch.empty_like(e1), torch.empty_like(e1), torch.empty_like(e1)
        for _ in range(3):
            dg.dftfe_chfsi_pass(made[0][1], X1, N, 12, b1, e1, r1, dg.DFTFE_MIXED_TF32X3)
            dg.dftfe_chfsi_pass(made[1][1], X2, N, 12, b2, e2, r2, dg.DFTFE_MIXED_TF32X3)
            torch.cuda.synchronize()
            assert torch.equal(X1, X2) and torch.equal(e1, e2)
        atmem, deep, deal, best, default = dg.dftfe_autotune_query_mixed(made[1][1])
        assert atmem in (0, 1) and deep in (0, 1) and deal in (0, 1) and 0.0 < best <= default
    finally:
        for mesh, ham in made:
            dg.dftfe_ham_destroy(ham)
            dg.dftfe_mesh_destroy(mesh)


def test_tuned_batch_of_shared_kpoints_is_bit_identical(dg):
    """Two systems x three k-points, the k-point hams of each system sharing its local
    operator, in tuned and untuned batches (TF32x3) and as single passes: all bit-identical;
    the tuner records one shape per distinct launch, the interleaved work list among the
    candidates."""
    systems = [_case(seed=7, n=(3, 3, 3), p=4, L=7.0), _case(seed=8, n=(2, 3, 2), p=4, L=6.0)]
    owners, hams = [], []
    for c in systems:
        mesh, src = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], None)
        owners.append((mesh, src))
        for k in KPTS:
            h = dg.dftfe_ham_create_shared(src)
            _kham(dg, c, mesh, h, k)
            hams.append((c, mesh, h))
    b_plain = dg.dftfe_batch_create([h for _, _, h in hams])
    try:
        N, blk, deg = 10, 10, 6
        X0 = [_start(dg, dg.dftfe_mesh_info(m)[0], N, 70 + i) for i, (_, m, _) in enumerate(hams)]
        bd0 = [dg.dftfe_spectrum_bounds_z(h, 20, 9, N) for _, _, h in hams]
        runs = []
        for mode in ("plain", "tuned", "single"):
            Xs = [x.clone() for x in X0]
            bds = [dg.make_bounds(b.a, b.b, b.a0) for b in bd0]
            evs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in Xs]
            rss = [torch.empty_like(e) for e in evs]
            if mode == "tuned":
                dg.dftfe_batch_autotune(b_plain, True)
            for _ in range(2):
                if mode == "single":
                    for i, (_, _, h) in enumerate(hams):
                        dg.dftfe_chfsi_pass_z(h, Xs[i], blk, deg, bds[i], evs[i], rss[i], dg.DFTFE_MIXED_TF32X3)
                else:
                    dg.dftfe_batch_chfsi_pass(b_plain, Xs, [blk] * len(Xs), [deg] * len(Xs), bds, evs, rss,
                                              dg.DFTFE_MIXED_TF32X3)
            torch.cuda.synchronize()
            runs.append((Xs, evs))
            if mode == "tuned":
                tuned = dg.dftfe_batch_autotune_query(b_plain)
                assert len(tuned) >= 1
                for t in tuned:
                    assert t["nodes_per_cell"] == 125 and t["order"] in (0, 1) and 0.0 < t["best_ms"] <= t["default_ms"]
                dg.dftfe_batch_autotune(b_plain, False)
        for Xs, evs in runs[1:]:
            for i in range(len(hams)):
                assert torch.equal(Xs[i], runs[0][0][i]) and torch.equal(evs[i], runs[0][1][i]), i
    finally:
        dg.dftfe_batch_destroy(b_plain)
        for _, _, h in hams:
            dg.dftfe_ham_destroy(h)
        for mesh, src in owners:
            dg.dftfe_ham_destroy(src)
            dg.dftfe_mesh_destroy(mesh)
