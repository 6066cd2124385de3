"""The learned degree/bounds proposer end to end on small seeded SCF-like sequences, in the
precision form (TF32x3 passes): data from the solver's own cost-based degree search, training
on the GPU kernels, then held-out sequences run twice from the same state -- with the standard
rule (Lanczos bound at every potential change, a = theta_N, degree 40) and with the proposer
(standard rule as fallback).  Both must reach the generalised-residual tolerance at every
step; the proposer must need fewer Lanczos runs, no more filter applications and less time
(the residual checks and the Lanczos runs inside the timed region).  Measured on GB300 with
200 x 20 training sequences: 21 % fewer applications and 2.6x less time on held-out
sequences of this system, 20 % and 34 % on the 32^3-cell, 1,024-state system."""
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
    replaces the Lanczos run at each potential change, needs no more filter applications and
    less time than the standard rule.  The comparison is printed."""
    dg, degree, wl, mesh, ham, qxyz = env
    prec = dg.DFTFE_MIXED_TF32X3
    steps, nseq = 8, 12
    F, T = [], []
    for seed in range(nseq):
        X = _start(dg, wl, seed)
        ctrl = degree.Controller(ham, wl.nstates, None, seed)
        stats, samples = degree.run_sequence(dg, ham, wl, qxyz, X, ctrl, seed, steps, TOL, prec=prec, search=True)
        assert all(s["max_resid"] <= TOL for s in stats)
        F += [s[0] for s in samples]
        T += [s[1] for s in samples]
    assert len(F) == nseq * steps
    net = degree.Network(seed=1)
    hist = net.train(np.array(F), np.array(T), steps=2000)
    assert hist[-1] < 0.1 * hist[0]
    tot = {n: {"applications": 0, "passes": 0, "seconds": 0.0, "lanczos": 0} for n in ("standard", "learned")}
    for seed in (100, 101, 102):
        for name, n in (("standard", None), ("learned", net)):
            X = _start(dg, wl, seed)
            ctrl = degree.Controller(ham, wl.nstates, n, seed)
            stats, _ = degree.run_sequence(dg, ham, wl, qxyz, X, ctrl, seed, steps, TOL, prec=prec)
            assert all(s["max_resid"] <= TOL for s in stats), (name, stats)
            tot[name]["applications"] += sum(s["applications"] for s in stats[1:])
            tot[name]["passes"] += sum(s["passes"] for s in stats[1:])
            tot[name]["seconds"] += sum(s["seconds"] for s in stats[1:])
            tot[name]["lanczos"] += ctrl.lanczos_runs
    with capsys.disabled():
        print(f"\nlearned proposer vs standard rule (3 held-out sequences x {steps} potentials):", tot)
    assert tot["learned"]["lanczos"] < tot["standard"]["lanczos"]
    assert tot["learned"]["applications"] <= tot["standard"]["applications"]
    assert tot["learned"]["seconds"] < tot["standard"]["seconds"]
