"""The learned degree/bounds proposer end to end on small seeded SCF-like sequences: data
from the solver's own degree search, training on the GPU kernels, then held-out sequences
run twice from the same state -- with the standard rule (Lanczos bound at every potential
change, a = theta_N, degree 40) and with the proposer (standard rule as fallback).  Both
must reach the residual tolerance at every step; the comparison is printed."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    from paper_2203_07820_gb300 import degree
    wl = synth.small_wells(0)
    mesh = dg.dftfe_mesh_create(wl.L, wl.ncell, wl.degree)
    ham = dg.dftfe_ham_create(mesh)
    _, qxyz = dg.dftfe_mesh_coords(mesh, nodes=False)
    yield dg, degree, wl, mesh, ham, qxyz
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)


def _start(dg, wl, seed):
    X = torch.empty((wl.ndofs, wl.nstates), dtype=torch.float64, device="cuda")
    dg.dftfe_random_uniform(X, 1000 + seed)
    return X


def test_learned_proposer_against_the_standard_rule(env, capsys):
    """Both controllers meet the tolerance at every step of held-out sequences; the proposer
    replaces the Lanczos run at each potential change and stays within 25 % of the standard
    rule's filter applications.  The comparison is printed (applications, passes, seconds)."""
    dg, degree, wl, mesh, ham, qxyz = env
    steps = 6
    F, T = [], []
    for seed in range(8):
        X = _start(dg, wl, seed)
        ctrl = degree.Controller(ham, wl.nstates, None, seed)
        stats, samples = degree.run_sequence(dg, ham, wl, qxyz, X, ctrl, seed, steps, TOL, search=True)
        assert all(s["max_resid"] <= TOL for s in stats)
        F += [s[0] for s in samples]
        T += [s[1] for s in samples]
    assert len(F) == 8 * steps
    net = degree.Network(seed=1)
    hist = net.train(np.array(F), np.array(T), steps=2000)
    assert hist[-1] < 0.1 * hist[0]
    tot = {n: {"applications": 0, "passes": 0, "seconds": 0.0, "lanczos": 0} for n in ("standard", "learned")}
    for seed in (100, 101, 102):
        for name, n in (("standard", None), ("learned", net)):
            X = _start(dg, wl, seed)
            ctrl = degree.Controller(ham, wl.nstates, n, seed)
            stats, _ = degree.run_sequence(dg, ham, wl, qxyz, X, ctrl, seed, steps, TOL)
            assert all(s["max_resid"] <= TOL for s in stats), (name, stats)
            tot[name]["applications"] += sum(s["applications"] for s in stats[1:])
            tot[name]["passes"] += sum(s["passes"] for s in stats[1:])
            tot[name]["seconds"] += sum(s["seconds"] for s in stats[1:])
            tot[name]["lanczos"] += ctrl.lanczos_runs
    with capsys.disabled():
        print("\nlearned proposer vs standard rule (3 held-out sequences x 6 potentials):", tot)
    assert tot["learned"]["lanczos"] < tot["standard"]["lanczos"]
    assert tot["learned"]["applications"] <= 1.25 * tot["standard"]["applications"]
