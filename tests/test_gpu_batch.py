"""Batched passes over independent systems of uneven mesh size, degree, state count and block
size: every system's result must be bit-identical to a pass of that system alone (same
operations in the same order), over two consecutive passes, and every item (Gamma point and
k-point) must match two passes of the FP64 oracle; a timing comparison on sixteen small
systems is printed."""
import math
import time

import numpy as np
import pytest

import oracle
import synth
from oracle import kpoint
from systems import gpu_system, oracle_system, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (seed, cells, p, L, nonlocal, states, block, degree, scaled)
SYSTEMS = [
    (0, (3, 3, 3), 4, 6.0, True, 20, 8, 9, True),      # last block of 4: narrow kernel alone
    (1, (4, 3, 2), 4, 8.0, False, 24, 24, 12, False),
    (2, (2, 2, 3), 6, 7.0, True, 37, 16, 7, True),
    (3, (4, 4, 4), 3, 8.0, False, 16, 7, 10, True),
    (4, (2, 3, 2), 5, 6.0, True, 30, 30, 0, True),      # degree 0: no filter
]


def _make(dg, spec):
    seed, n, p, L, nl, N, block, deg, scaled = spec
    c = small_case(seed, n=n, p=p, L=L, nl=nl)
    mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    M = dg.dftfe_mesh_info(mesh)[0]
    X = torch.empty((M, N), dtype=torch.float64, device="cuda")
    dg.dftfe_random_uniform(X, 100 + seed)
    bd = dg.dftfe_spectrum_bounds(ham, 20, 7 + seed, N)
    if not scaled:
        bd = dg.make_bounds(bd.a, bd.b)
    return mesh, ham, X, bd, block, deg


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


def test_batched_passes_are_bit_identical_to_single_passes(dg):
    made = [_make(dg, s) for s in SYSTEMS]
    hams = [m[1] for m in made]
    batch = dg.dftfe_batch_create(hams)
    try:
        Xb = [m[2].clone() for m in made]
        Xs = [m[2].clone() for m in made]
        bb = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made]
        bs = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made]
        evb = [torch.empty(x.shape[1], dtype=torch.float64, device="cuda") for x in Xb]
        rsb = [torch.empty_like(e) for e in evb]
        evs = [torch.empty_like(e) for e in evb]
        rss = [torch.empty_like(e) for e in evb]
        blocks = [m[4] for m in made]
        degs = [m[5] for m in made]
        for _ in range(2):
            dg.dftfe_batch_chfsi_pass(batch, Xb, blocks, degs, bb, evb, rsb)
            for i, (mesh, ham, _, _, block, deg) in enumerate(made):
                dg.dftfe_chfsi_pass(ham, Xs[i], block, deg, bs[i], evs[i], rss[i])
            torch.cuda.synchronize()
            for i in range(len(made)):
                assert torch.equal(Xb[i], Xs[i]), i
                assert torch.equal(evb[i], evs[i]) and torch.equal(rsb[i], rss[i]), i
                for f in ("a", "b", "a0"):
                    x, y = getattr(bb[i], f), getattr(bs[i], f)
                    assert x == y or (math.isnan(x) and math.isnan(y)), (i, f)
    finally:
        dg.dftfe_batch_destroy(batch)
        for mesh, ham, *_ in made:
            dg.dftfe_ham_destroy(ham)
            dg.dftfe_mesh_destroy(mesh)


def test_batch_rejects_bad_input(dg):
    spec = SYSTEMS[1]
    mesh, ham, X, bd, block, deg = _make(dg, spec)
    try:
        with pytest.raises(dg.DftfeError):
            dg.dftfe_batch_create([ham, ham])                      # duplicate
        batch = dg.dftfe_batch_create([ham])
        ev = torch.empty(X.shape[1], dtype=torch.float64, device="cuda")
        rs = torch.empty_like(ev)
        with pytest.raises(dg.DftfeError):
            dg.dftfe_batch_chfsi_pass(batch, [X], [block], [deg], [dg.make_bounds(bd.b, bd.a)], [ev], [rs])
        with pytest.raises(dg.DftfeError):
            dg.dftfe_batch_chfsi_pass(batch, [X], [block], [deg], [bd], [ev], [rs], prec=dg.DFTFE_MIXED_BF16X3)
        dg.dftfe_batch_destroy(batch)
    finally:
        dg.dftfe_ham_destroy(ham)
        dg.dftfe_mesh_destroy(mesh)


def test_batch_of_sixteen_small_systems_timing(dg, capsys):
    specs = []
    for i in range(16):
        n = (3 + i % 3, 3 + (i // 3) % 3, 3 + (i // 9) % 2)
        specs.append((i, n, 4 + i % 3, 6.0 + n[0], i % 2 == 0, 16 + 8 * (i % 4), 16, 20 + 4 * (i % 6), True))
    made = [_make(dg, s) for s in specs]
    batch = dg.dftfe_batch_create([m[1] for m in made])
    try:
        def run(batched):
            Xs = [m[2].clone() for m in made]
            bds = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made]
            evs = [torch.empty(x.shape[1], dtype=torch.float64, device="cuda") for x in Xs]
            rss = [torch.empty_like(e) for e in evs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if batched:
                dg.dftfe_batch_chfsi_pass(batch, Xs, [m[4] for m in made], [m[5] for m in made], bds, evs, rss)
            else:
                for i, m in enumerate(made):
                    dg.dftfe_chfsi_pass(m[1], Xs[i], m[4], m[5], bds[i], evs[i], rss[i])
            torch.cuda.synchronize()
            return time.perf_counter() - t0, Xs
        run(True), run(False)                                   # warm-up
        tb, xb = run(True)
        ts, xs = run(False)
        assert all(torch.equal(a, b) for a, b in zip(xb, xs))
        dg.dftfe_batch_use_graphs(batch, True)
        run(True)                                               # first graphed pass runs directly
        tg, xg = run(True)
        assert all(torch.equal(a, b) for a, b in zip(xg, xs))
        for m in made:
            dg.dftfe_profile_enable(m[1], True)
        run(True)
        filt = dg.dftfe_profile_query(made[0][1], "batch_filter")[0]
        chol = sum(dg.dftfe_profile_query(m[1], "pass_cholgs")[0] for m in made)
        rr = sum(dg.dftfe_profile_query(m[1], "pass_rr")[0] for m in made)
        for m in made:
            dg.dftfe_profile_enable(m[1], False)
        with capsys.disabled():
            print(f"\n16 systems ({sum(m[2].shape[0] for m in made)} DoFs in all): batched pass {tb * 1e3:.1f} ms, "
                  f"graphed {tg * 1e3:.1f} ms, one by one {ts * 1e3:.1f} ms; batched phases: filter {filt:.1f} ms, "
                  f"CholGS {chol:.1f} ms, Rayleigh-Ritz {rr:.1f} ms")
    finally:
        dg.dftfe_batch_destroy(batch)
        for mesh, ham, *_ in made:
            dg.dftfe_ham_destroy(ham)
            dg.dftfe_mesh_destroy(mesh)


# (seed, cells, p, L, states, block, degree, k)
KSYSTEMS = [
    (0, (3, 3, 3), 4, 6.0, 12, 5, 9, (0.2, -0.1, 0.3)),
    (0, (3, 3, 3), 4, 6.0, 12, 5, 9, (math.pi / 6.0, 0.0, 0.0)),   # a second k-point of the same system
    (2, (2, 2, 3), 6, 7.0, 10, 2, 7, (0.0, 0.4, 0.0)),              # 2-column blocks: narrow kernel alone
    (3, (4, 3, 2), 5, 8.0, 16, 16, 8, (0.1, 0.1, 0.1)),
]


def _make_k(dg, spec):
    seed, n, p, L, N, block, deg, k = spec
    c = small_case(seed, n=n, p=p, L=L, nl=True)
    mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    nxyz, _ = dg.dftfe_mesh_coords(mesh, quad=False)
    cent, w, rc, hc = c["proj"]
    dg.dftfe_ham_set_kpoint(ham, k, synth.projector_disp(nxyz, cent, rc, c["L"]))
    M = nxyz.shape[0]
    Xr = torch.empty((M, 2 * N), dtype=torch.float64, device="cuda")
    dg.dftfe_random_uniform(Xr, 300 + seed)
    bd = dg.dftfe_spectrum_bounds_z(ham, 20, 9 + seed, N)
    return mesh, ham, Xr.view(torch.complex128), bd, block, deg


def test_batched_kpoint_and_gamma_passes_are_bit_identical(dg):
    """Complex items at k-points (two k-points of one system among them) and real Gamma-point
    items in one batch: each result equals the pass of that item alone."""
    made = [_make_k(dg, s) for s in KSYSTEMS] + [_make(dg, SYSTEMS[1]), _make(dg, SYSTEMS[2])]
    batch = dg.dftfe_batch_create([m[1] for m in made])
    try:
        Xb = [m[2].clone() for m in made]
        Xs = [m[2].clone() for m in made]
        bb = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made]
        bs = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made]
        evb = [torch.empty(x.shape[1], dtype=torch.float64, device="cuda") for x in Xb]
        rsb = [torch.empty_like(e) for e in evb]
        evs = [torch.empty_like(e) for e in evb]
        rss = [torch.empty_like(e) for e in evb]
        for _ in range(2):
            dg.dftfe_batch_chfsi_pass(batch, Xb, [m[4] for m in made], [m[5] for m in made], bb, evb, rsb)
            for i, (mesh, ham, X0, _, block, deg) in enumerate(made):
                if X0.is_complex():
                    dg.dftfe_chfsi_pass_z(ham, Xs[i], block, deg, bs[i], evs[i], rss[i])
                else:
                    dg.dftfe_chfsi_pass(ham, Xs[i], block, deg, bs[i], evs[i], rss[i])
            torch.cuda.synchronize()
            for i in range(len(made)):
                assert torch.equal(Xb[i], Xs[i]), i
                assert torch.equal(evb[i], evs[i]) and torch.equal(rsb[i], rss[i]), i
        # the two k-points of the same system differ (the k terms are there)
        assert not torch.equal(evb[0], evb[1])
    finally:
        dg.dftfe_batch_destroy(batch)
        for mesh, ham, *_ in made:
            dg.dftfe_ham_destroy(ham)
            dg.dftfe_mesh_destroy(mesh)


def test_batch_of_systems_times_kpoints_timing(dg, capsys):
    """Four small systems x four k-points each in one batched pass against one by one."""
    specs = []
    for i in range(4):
        n = (3 + i % 2, 3, 3 + i // 2)
        for q in range(4):
            k = (0.5 * q / (6.0 + n[0]), 0.1 * q, -0.05 * q)
            specs.append((i, n, 4 + i % 3, 6.0 + n[0], 16, 16, 16, k))
    made = [_make_k(dg, s) for s in specs]
    batch = dg.dftfe_batch_create([m[1] for m in made])
    try:
        def run(batched):
            Xs = [m[2].clone() for m in made]
            bds = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made]
            evs = [torch.empty(x.shape[1], dtype=torch.float64, device="cuda") for x in Xs]
            rss = [torch.empty_like(e) for e in evs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if batched:
                dg.dftfe_batch_chfsi_pass(batch, Xs, [m[4] for m in made], [m[5] for m in made], bds, evs, rss)
            else:
                for i, m in enumerate(made):
                    dg.dftfe_chfsi_pass_z(m[1], Xs[i], m[4], m[5], bds[i], evs[i], rss[i])
            torch.cuda.synchronize()
            return time.perf_counter() - t0, Xs
        run(True), run(False)
        tb, xb = run(True)
        ts, xs = run(False)
        assert all(torch.equal(a, b) for a, b in zip(xb, xs))
        with capsys.disabled():
            print(f"\n4 systems x 4 k-points (complex128): batched pass {tb * 1e3:.1f} ms, one by one {ts * 1e3:.1f} ms")
    finally:
        dg.dftfe_batch_destroy(batch)
        for mesh, ham, *_ in made:
            dg.dftfe_ham_destroy(ham)
            dg.dftfe_mesh_destroy(mesh)


def test_graphed_batched_pass_is_bit_identical(dg):
    """The batched filter phase as one CUDA graph (Gamma-point and k-point items, a narrow
    block among them) gives the bits of the plain batched pass."""
    specs = [SYSTEMS[0], SYSTEMS[2]]
    made1 = [_make(dg, s) for s in specs] + [_make_k(dg, KSYSTEMS[0]), _make_k(dg, KSYSTEMS[2])]
    made2 = [_make(dg, s) for s in specs] + [_make_k(dg, KSYSTEMS[0]), _make_k(dg, KSYSTEMS[2])]
    b1 = dg.dftfe_batch_create([m[1] for m in made1])
    b2 = dg.dftfe_batch_create([m[1] for m in made2])
    dg.dftfe_batch_use_graphs(b2, True)
    try:
        X1 = [m[2].clone() for m in made1]
        X2 = [m[2].clone() for m in made1]
        bd1 = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made1]
        bd2 = [dg.make_bounds(m[3].a, m[3].b, m[3].a0) for m in made1]
        e1 = [torch.empty(x.shape[1], dtype=torch.float64, device="cuda") for x in X1]
        r1 = [torch.empty_like(e) for e in e1]
        e2 = [torch.empty_like(e) for e in e1]
        r2 = [torch.empty_like(e) for e in e1]
        blocks, degs = [m[4] for m in made1], [m[5] for m in made1]
        for it in range(3):
            dg.dftfe_batch_chfsi_pass(b1, X1, blocks, degs, bd1, e1, r1)
            dg.dftfe_batch_chfsi_pass(b2, X2, blocks, degs, bd2, e2, r2)
            torch.cuda.synchronize()
            for i in range(len(X1)):
                assert torch.equal(X1[i], X2[i]) and torch.equal(e1[i], e2[i]), (it, i)
        assert dg.dftfe_batch_graph_query(b2)[0] == 2
    finally:
        dg.dftfe_batch_destroy(b1)
        dg.dftfe_batch_destroy(b2)
        for mesh, ham, *_ in made1 + made2:
            dg.dftfe_ham_destroy(ham)
            dg.dftfe_mesh_destroy(mesh)


def _oracle_gamma(spec):
    seed, n, p, L, nl, N, block, deg, scaled = spec
    c = small_case(seed, n=n, p=p, L=L, nl=nl)
    om, oh = oracle_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    tmin, _, b = oracle.lanczos_bounds(oh.apply, synth.counter_uniform(7 + seed, om.ndofs), 20)
    bd = oracle.first_pass_bounds(tmin, b, N, om.ndofs)
    if not scaled:
        bd = oracle.Bounds(bd.a, bd.b)
    return c, om, oh, synth.random_block(100 + seed, om.ndofs, N), bd


def _oracle_kpoint(spec):
    seed, n, p, L, N, block, deg, k = spec
    c = small_case(seed, n=n, p=p, L=L, nl=True)
    om, oh = oracle_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], None)
    bh = kpoint.BlochHamiltonian(oh, k)
    cent, w, rc, hc = c["proj"]
    rp, nd, chi = synth.projector_csr(om.node_xyz(), cent, w, rc, c["L"])
    bh.set_nonlocal(hc, rp, nd, chi, synth.projector_disp(om.node_xyz(), cent, rc, c["L"]))
    tmin, _, b = kpoint.spectrum_bounds(bh, synth.counter_uniform(9 + seed, 2 * om.ndofs), 20)
    bd = oracle.first_pass_bounds(tmin, b, N, om.ndofs)
    Z0 = synth.random_block(300 + seed, om.ndofs, 2 * N).view(np.complex128)
    return c, om, bh, Z0, bd


def test_batched_passes_match_the_oracle(dg):
    """Every item of a batch (five Gamma-point systems -- degree 0, blocks of 7 and 30, a
    narrow-kernel tail -- and four k-point items, two of them k-points of one system) against
    two passes of the FP64 oracles from the same seeded start and the oracle's own bounds:
    Ritz values within 1e-9 Ha and the same bounds updates."""
    items = []
    for spec in SYSTEMS:
        c, om, oh, X0, bd = _oracle_gamma(spec)
        mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
        items.append(dict(mesh=mesh, ham=ham, X=torch.from_numpy(X0).cuda(), X0=X0, bd=bd, oracle=oh, cplx=False,
                          block=spec[6], deg=spec[7]))
    for spec in KSYSTEMS:
        c, om, bh, Z0, bd = _oracle_kpoint(spec)
        mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
        nxyz, _ = dg.dftfe_mesh_coords(mesh, quad=False)
        cent, w, rc, hc = c["proj"]
        dg.dftfe_ham_set_kpoint(ham, spec[7], synth.projector_disp(nxyz, cent, rc, c["L"]))
        items.append(dict(mesh=mesh, ham=ham, X=torch.from_numpy(Z0.copy()).cuda(), X0=Z0, bd=bd, oracle=bh,
                          cplx=True, block=spec[5], deg=spec[6]))
    batch = dg.dftfe_batch_create([it["ham"] for it in items])
    try:
        gbs = [dg.make_bounds(it["bd"].a, it["bd"].b, it["bd"].a0) for it in items]
        evs = [torch.empty(it["X"].shape[1], dtype=torch.float64, device="cuda") for it in items]
        rss = [torch.empty_like(e) for e in evs]
        Xo = [it["X0"] for it in items]
        obs = [it["bd"] for it in items]
        for _ in range(2):
            dg.dftfe_batch_chfsi_pass(batch, [it["X"] for it in items], [it["block"] for it in items],
                                      [it["deg"] for it in items], gbs, evs, rss)
            torch.cuda.synchronize()
            for i, it in enumerate(items):
                run = kpoint.chfsi_pass if it["cplx"] else oracle.chfsi_pass
                Xo[i], _, theta, _, obs[i] = run(it["oracle"], Xo[i], it["block"], it["deg"], obs[i])
                assert np.abs(evs[i].cpu().numpy() - theta).max() < 1e-9, i
                assert abs(gbs[i].a - obs[i].a) < 1e-9, i
                assert (math.isnan(gbs[i].a0) and math.isnan(obs[i].a0)) or abs(gbs[i].a0 - obs[i].a0) < 1e-9, i
    finally:
        dg.dftfe_batch_destroy(batch)
        for it in items:
            dg.dftfe_ham_destroy(it["ham"])
            dg.dftfe_mesh_destroy(it["mesh"])


def test_batched_tf32x3_passes_are_bit_identical_and_match_the_oracle(dg):
    """The split-precision batched pass (one persistent cell-product launch per step and degree
    over every system's cells): Gamma-point items of degrees p = 4, 6, 3 (degree 0 among them,
    blocks of 7, 8, 16, 24 and 30) and k-point items (complex64) give the bits of single TF32x3
    passes, over two passes; and after twelve passes the Ritz values of the lower half of every
    item are within 1e-6 Ha of twelve FP64 oracle passes from the same start."""
    items = []
    for spec in SYSTEMS:
        c, om, oh, X0, bd = _oracle_gamma(spec)
        made = [gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
                for _ in range(2)]
        items.append(dict(sys=made, X0=X0, bd=bd, oracle=oh, cplx=False, block=spec[6], deg=spec[7]))
    for spec in KSYSTEMS:
        c, om, bh, Z0, bd = _oracle_kpoint(spec)
        made = []
        for _ in range(2):
            mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
            nxyz, _ = dg.dftfe_mesh_coords(mesh, quad=False)
            cent, w, rc, hc = c["proj"]
            dg.dftfe_ham_set_kpoint(ham, spec[7], synth.projector_disp(nxyz, cent, rc, c["L"]))
            made.append((mesh, ham))
        items.append(dict(sys=made, X0=Z0, bd=bd, oracle=bh, cplx=True, block=spec[5], deg=spec[6]))
    prec = dg.DFTFE_MIXED_TF32X3
    batch = dg.dftfe_batch_create([it["sys"][0][1] for it in items])
    try:
        Xb = [torch.from_numpy(it["X0"].copy()).cuda() for it in items]
        Xs = [x.clone() for x in Xb]
        bb = [dg.make_bounds(it["bd"].a, it["bd"].b, it["bd"].a0) for it in items]
        bs = [dg.make_bounds(it["bd"].a, it["bd"].b, it["bd"].a0) for it in items]
        evb = [torch.empty(x.shape[1], dtype=torch.float64, device="cuda") for x in Xb]
        rsb = [torch.empty_like(e) for e in evb]
        evs = [torch.empty_like(e) for e in evb]
        rss = [torch.empty_like(e) for e in evb]
        Xo = [it["X0"] for it in items]
        obs = [it["bd"] for it in items]
        thetas = [None] * len(items)
        for p_ in range(12):
            dg.dftfe_batch_chfsi_pass(batch, Xb, [it["block"] for it in items], [it["deg"] for it in items], bb,
                                      evb, rsb, prec)
            for i, it in enumerate(items):
                ham = it["sys"][1][1]
                if p_ < 2 and it["cplx"]:
                    dg.dftfe_chfsi_pass_z(ham, Xs[i], it["block"], it["deg"], bs[i], evs[i], rss[i], prec)
                elif p_ < 2:
                    dg.dftfe_chfsi_pass(ham, Xs[i], it["block"], it["deg"], bs[i], evs[i], rss[i], prec)
                run = kpoint.chfsi_pass if it["cplx"] else oracle.chfsi_pass
                Xo[i], _, thetas[i], _, obs[i] = run(it["oracle"], Xo[i], it["block"], it["deg"], obs[i])
            torch.cuda.synchronize()
            for i in range(len(items)):
                if p_ < 2:
                    assert torch.equal(Xb[i], Xs[i]), (p_, i)
                    assert torch.equal(evb[i], evs[i]) and torch.equal(rsb[i], rss[i]), (p_, i)
        for i, it in enumerate(items):
            if it["deg"] == 0:          # never filtered: not the mixed scheme's converged regime
                continue
            n2 = evb[i].shape[0] // 2
            assert np.abs(evb[i].cpu().numpy()[:n2] - thetas[i][:n2]).max() < 1e-6, i
    finally:
        dg.dftfe_batch_destroy(batch)
        for it in items:
            for mesh, ham in it["sys"]:
                dg.dftfe_ham_destroy(ham)
                dg.dftfe_mesh_destroy(mesh)
