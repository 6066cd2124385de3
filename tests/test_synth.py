"""Pins for the shared seeded-input module (SplitMix64 and the model functions)."""
import os
import numpy as np
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_u64():
    vals = []
    for line in open(os.path.join(GOLD, "splitmix64.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            vals.append(int(line, 16))
    return vals


def test_splitmix64_reference_outputs():
    ref = _golden_u64()
    # counter mode with seed 0: u64(idx) = mix((idx+1) * GAMMA) is the idx-th stream output
    z = np.arange(1, 4, dtype=np.uint64) * np.uint64(synth.GAMMA)
    got = [int(v) for v in synth._mix_u64(z)]
    assert got == ref
    assert [synth._mix_int(((i + 1) * synth.GAMMA) & synth.MASK) for i in range(3)] == ref
    s = synth.Stream(0 ^ synth.STREAM_XOR)   # state 0
    assert [s.next_u64() for _ in range(3)] == ref


def test_counter_uniform_range_and_layout():
    u = synth.counter_uniform(7, 10000)
    assert u.min() >= -0.5 and u.max() < 0.5
    assert abs(u.mean()) < 0.01
    X = synth.random_block(7, 100, 100)
    assert np.array_equal(X.ravel(), u)
    # offset counter continues the same sequence
    assert np.array_equal(synth.counter_uniform(7, 10, 95), u[95:105])


def test_gaussian_wells_single_atom():
    L = 40.0
    pts = np.array([[20.0, 20.0, 20.0], [21.0, 20.0, 20.0], [20.0, 22.0, 21.0], [0.5, 0.5, 0.5]])
    v = synth.gaussian_wells(pts, [[20.0, 20.0, 20.0]], 2.0, 1.0, L)
    r2 = np.sum((pts - 20.0) ** 2, axis=1)
    ref = np.where(r2 < 64.0, -2.0 * np.exp(-r2 / 2.0), 0.0)
    assert np.allclose(v, ref, rtol=0, atol=1e-15)


def test_gaussian_wells_periodic():
    L = 10.0
    c = [[1.0, 2.0, 3.0]]
    pts = np.random.default_rng(0).uniform(0, L, (50, 3))
    v = synth.gaussian_wells(pts, c, 2.0, 1.0, L)
    v2 = synth.gaussian_wells(pts + L * np.array([1, -2, 3]), c, 2.0, 1.0, L)
    assert np.allclose(v, v2, atol=1e-13)


def test_projector_csr_shapes():
    xyz = np.random.default_rng(1).uniform(0, 10, (2000, 3))
    rowptr, node, chi = synth.projector_csr(xyz, [[5, 5, 5], [1, 1, 1]], 1.0, 3.0, 10.0)
    assert rowptr.size == 9 and rowptr[-1] == node.size == chi.size
    for a in range(2):
        counts = np.diff(rowptr[4 * a:4 * a + 5])
        assert np.all(counts == counts[0])


def test_workload_recipes():
    w0 = synth.small_wells(0)
    assert w0.ndofs == 13824 and w0.centres.shape == (8, 3)
    assert np.all((w0.centres >= 0) & (w0.centres < 10))
    w1 = synth.lattice_atoms(0)
    assert w1.ndofs == 2985984 and w1.centres.shape == (64, 3) and w1.nproj == 256
    site = (np.arange(4) + 0.5) * 7.5
    assert np.all(np.abs(w1.centres[:4, 0] - site) <= 0.5)
    assert np.all((w1.couplings >= 0.5) & (w1.couplings <= 2.0))


def test_projector_disp_matches_the_csr_entries():
    """Each displacement reproduces its CSR entry's projector value (same order, minimum
    image, per-axis box lengths)."""
    import math
    L = np.array([6.0, 7.0, 8.0])
    s = synth.Stream(4)
    pts = np.array([[L[d] * s.uniform() for d in range(3)] for _ in range(400)])
    cent = np.array([[0.2, 6.8, 4.0], [5.9, 0.1, 7.9]])
    w, rc = 1.0, 2.5
    rowptr, node, chi = synth.projector_csr(pts, cent, w, rc, L)
    disp = synth.projector_disp(pts, cent, rc, L)
    assert disp.shape == (node.size, 3)
    n_s = (math.pi * w * w) ** 0.75
    n_p = math.sqrt(0.5 * (math.pi * w * w) ** 1.5)
    for a in range(len(cent)):
        for j in range(4):
            e0, e1 = rowptr[4 * a + j], rowptr[4 * a + j + 1]
            d = disp[e0:e1]
            # the displacement is the minimum image of node - centre
            raw = pts[node[e0:e1]] - cent[a]
            assert np.allclose(d, raw - L * np.round(raw / L))
            r2 = np.einsum("ij,ij->i", d, d)
            assert np.all(r2 < rc * rc)
            g = np.exp(-r2 / (2 * w * w))
            ref = g / n_s if j == 0 else (d[:, j - 1] / w) * g / n_p
            assert np.allclose(chi[e0:e1], ref, rtol=1e-14, atol=1e-300)


def test_kpoint_batch_recipe_spans_the_stated_ranges():
    """The batched k-point workload: sixteen systems of 8^3-20^3 cells, p = 4-6, 64-768 states,
    8-48 atoms with 4 projectors each, Chebyshev degrees 20-40; every system carries the 8
    points of the 2 x 2 x 2 Monkhorst-Pack grid (2 pi / L)(+-1/4, +-1/4, +-1/4), all inside
    the first Brillouin zone, distinct and summing to zero; atoms inside the box; seeds give
    distinct systems and repeat exactly."""
    import math
    out = synth.kpoint_batch(0)
    assert len(out) == 16
    cells = [wl.ncell for wl, _ in out]
    ps = [wl.degree for wl, _ in out]
    states = [wl.nstates for wl, _ in out]
    atoms = [len(wl.centres) for wl, _ in out]
    degs = [wl.cheb_degree for wl, _ in out]
    assert (min(cells), max(cells)) == (8, 20) and set(ps) == {4, 5, 6}
    assert (min(states), max(states)) == (64, 768) and (min(atoms), max(atoms)) == (8, 48)
    assert (min(degs), max(degs)) == (20, 40)
    for wl, kpts in out:
        assert wl.couplings.size == 4 * len(wl.centres)
        assert np.all((wl.centres >= 0.0) & (wl.centres < wl.L))
        assert np.all((wl.couplings >= 0.5) & (wl.couplings <= 2.0))
        assert wl.proj_cutoff < wl.L / 2          # minimum image is the only image
        k = np.array(kpts)
        assert k.shape == (8, 3) and len({tuple(v) for v in k}) == 8
        assert np.allclose(np.abs(k), 0.5 * math.pi / wl.L)
        assert np.allclose(k.sum(axis=0), 0.0)
    again = synth.kpoint_batch(0)
    assert all(np.array_equal(a.centres, b.centres) for (a, _), (b, _) in zip(out, again))
    other = synth.kpoint_batch(1)
    assert not np.array_equal(out[0][0].centres, other[0][0].centres)
