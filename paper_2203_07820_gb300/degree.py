"""Learned Chebyshev degree and unwanted-interval bounds for the next ChFSI pass.

The standard rule estimates the upper bound b of H~ with a k-step Lanczos run whenever the
Hamiltonian changes, cuts the unwanted interval at a = theta_N (the largest Ritz value of the
previous pass) and filters with a fixed degree (40 here).  The learned proposer replaces
that with a three-layer FP32 network evaluated by the library's kernels (dftfe_mlp_*): from
the last three passes' residual statistics, spectrum spread, bounds and degrees it proposes
the next degree, where the largest wanted Ritz value will move (a) and the ratio of the new
upper bound to the last one (b), so no Lanczos run is needed when the potential changes.
The standard rule stays in charge of the first potential of a sequence and of the rest of a
potential after a proposed pass that failed to halve the largest residual; it also judges
the proposer.

Training targets come from the solver itself (`search_step`): at a potential change, passes
with each candidate degree and the standard bounds are run from a copy of the state until the
tolerance is met, each roll-out timed on the GPU, and the target is the degree with the least
time to the tolerance (its filter applications plus the fixed orthonormalisation and
projection cost of every pass it needs; fewer applications break near-ties).  Inputs: seeded
sequences of potentials whose atoms move 0.05 bohr per step, mixed 0.3 old / 0.7 new.

Host logic only chooses parameters; the passes, the Lanczos runs and the network run on the
GPU through the C ABI.
"""
import math
import time

import numpy as np

from . import (dftfe_chfsi_pass, dftfe_lanczos, dftfe_mlp_adam, dftfe_mlp_forward, dftfe_mlp_loss_grad,
               dftfe_mlp_param_count, dftfe_spectrum_bounds, make_bounds)

N_IN, N_H, N_OUT = 19, 64, 3
SHAPE = (N_IN, N_H, N_OUT)
FALLBACK_DEGREE = 40
CANDIDATES = (8, 12, 16, 20, 24, 32, 48)
LANCZOS_K = 20
B_MARGIN = 1.01            # safety factor on a proposed upper bound
DEG_MIN, DEG_MAX = 4, 64
CONVERGED_FRACTION = 0.75  # the lowest 3/4 of the states must meet the tolerance; the top
                           # quarter is the buffer that ChFSI carries to let them converge


class Record:
    """What one pass left behind (host copies of its Ritz values and residuals)."""

    def __init__(self, evals, resid, a, b, degree, first):
        self.evals = np.asarray(evals, dtype=np.float64)
        self.resid = np.asarray(resid, dtype=np.float64)
        self.a, self.b, self.degree, self.first = float(a), float(b), int(degree), bool(first)

    @property
    def rmax(self):
        """Largest residual over the states that must converge (the lowest 3/4)."""
        n = max(1, int(math.ceil(CONVERGED_FRACTION * self.resid.size)))
        return float(self.resid[:n].max())


class Judge:
    """The convergence test of the sequences: the largest generalised residual
    ||H psi - eps M psi|| / ||psi|| (psi = M^-1/2 x, the residual of the metric) over the
    lowest 3/4 of the states, from an FP64-accurate H~X -- the exact digit products on the
    tensor cores (the FP64 cell kernel beyond their degree range) -- in column chunks of 128,
    so the test needs two M x 128 buffers, not a second block.  The same test, with its time,
    for every precision and controller.  (The passes' own Loewdin residual ||H~x - theta x||
    is larger by the inverse lumped mass, 10 to 500 times on the test meshes, and has the FP32
    filter's noise floor, about lambda_max 2^-24, at the 1e-5 tolerance.)"""

    CHUNK = 128

    def __init__(self):
        self._fp64 = set()
        self._buf = {}

    def _apply(self, ham, x, w):
        from . import DFTFE_FP64, DFTFE_FP64_SLICES, DftfeError, dftfe_ham_apply
        key = id(ham)
        if key not in self._fp64:
            try:
                dftfe_ham_apply(ham, x, w, DFTFE_FP64_SLICES)
                return
            except DftfeError:
                self._fp64.add(key)
        dftfe_ham_apply(ham, x, w, DFTFE_FP64)

    def __call__(self, ham, X, ev):
        import torch
        from . import dftfe_residuals
        M, N = X.shape
        n = max(1, int(math.ceil(CONVERGED_FRACTION * N)))
        cw = min(self.CHUNK, n)
        key = (M, cw, str(X.device))
        if key not in self._buf:
            self._buf = {key: (torch.empty((M, cw), dtype=torch.float64, device=X.device),
                               torch.empty((M, cw), dtype=torch.float64, device=X.device),
                               torch.empty(cw, dtype=torch.float64, device=X.device))}
        xc, wc, rg = self._buf[key]
        worst = 0.0
        for j0 in range(0, n, cw):
            k = min(n, j0 + cw) - j0
            x, w = (xc, wc) if k == cw else (xc[:, :k], wc[:, :k])
            x.copy_(X[:, j0:j0 + k])
            self._apply(ham, x, w)
            dftfe_residuals(ham, x, w, ev[j0:j0 + k], rg[:k], 1)
            worst = max(worst, float(rg[:k].max().item()))
        return worst


def features(hist, first_next):
    """Input vector of the proposer for the pass after `hist` (a non-empty list of Records,
    most recent last): per pass (most recent first, the oldest repeated when fewer than
    three): log10 max and median residual (/4), spread (theta_N - theta_1)/(b - theta_1),
    cut position (a - theta_1)/(b - theta_1), degree/40, log(b / b_last); then a flag for
    'the potential changed before this pass'."""
    f = []
    last_b = hist[-1].b
    for j in range(3):
        r = hist[max(0, len(hist) - 1 - j)]
        t1, tn = r.evals[0], r.evals[-1]
        den = max(r.b - t1, 1e-12)
        f += [math.log10(max(r.rmax, 1e-30)) / 4.0, math.log10(max(float(np.median(r.resid)), 1e-30)) / 4.0,
              (tn - t1) / den, (r.a - t1) / den, r.degree / 40.0, math.log(max(r.b, 1e-12) / last_b)]
    f.append(1.0 if first_next else 0.0)
    return np.array(f, dtype=np.float64)


def decode(y, last, b_est):
    """Proposed (degree, a, b used, new upper-bound estimate) from network outputs
    y = (log2(m/16), drift of theta_N in units of the spectrum spread, log of the new-to-last
    upper-bound ratio).  The safety margin goes on the bound used, not on the estimate that
    the next proposal starts from, so it does not compound."""
    m = int(min(DEG_MAX, max(DEG_MIN, round(16.0 * 2.0 ** float(y[0])))))
    t1, tn = last.evals[0], last.evals[-1]
    spread = max(tn - t1, 1e-12)
    # the cut moves up with the predicted drift of theta_N, by at most 2 % of the spread
    # (a cut inside the wanted spectrum damps wanted states), never below theta_N
    a = tn + min(max(float(y[1]), 0.0), 0.02) * spread
    est = b_est * math.exp(min(max(float(y[2]), -0.02), 0.02))
    return m, a, max(est * B_MARGIN, a + spread), est


class Network:
    """The proposer's parameters on the GPU and the library kernels that use them."""

    def __init__(self, params=None, seed=0):
        import torch
        import synth
        self.torch = torch
        P = dftfe_mlp_param_count(*SHAPE)
        if params is None:
            u = synth.counter_uniform(seed, P) * 2.0       # U(-1, 1), scaled per layer below
            o = 0
            scale = np.empty(P)
            for rows, cols in ((N_H, N_IN), (N_H, None), (N_H, N_H), (N_H, None), (N_OUT, N_H), (N_OUT, None)):
                k = rows * (cols or 1)
                scale[o:o + k] = 1.0 / math.sqrt(cols) if cols else 0.0
                o += k
            params = u * scale
        self.params = torch.tensor(np.asarray(params, dtype=np.float32), device="cuda")
        self.mu = np.zeros(N_IN)
        self.sd = np.ones(N_IN)

    def predict(self, F):
        torch = self.torch
        Fz = (np.atleast_2d(F) - self.mu) / self.sd
        X = torch.tensor(Fz.astype(np.float32), device="cuda")
        Y = torch.empty((X.shape[0], N_OUT), dtype=torch.float32, device="cuda")
        dftfe_mlp_forward(self.params, SHAPE, X, Y)
        return Y.cpu().numpy().astype(np.float64)

    def train(self, F, T, weights=(1.0, 0.5, 1.0), steps=3000, lr=3e-3):
        """Full-batch Adam on the GPU kernels; inputs standardised with the training set's
        mean and spread (kept for prediction).  Returns the loss history (every 100 steps)."""
        torch = self.torch
        F = np.asarray(F, dtype=np.float64)
        self.mu = F.mean(axis=0)
        # a floor on the spread: a feature that barely varies in the training set must not
        # be blown up into a saturating input when it moves at inference
        self.sd = np.maximum(F.std(axis=0), 0.1)
        X = torch.tensor(((F - self.mu) / self.sd).astype(np.float32), device="cuda")
        Tt = torch.tensor(np.asarray(T, dtype=np.float32), device="cuda")
        w = torch.tensor(np.asarray(weights, dtype=np.float32), device="cuda")
        g = torch.empty_like(self.params)
        m = torch.zeros_like(self.params)
        v = torch.zeros_like(self.params)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        hist = []
        for t in range(1, steps + 1):
            dftfe_mlp_loss_grad(self.params, SHAPE, X, Tt, w, loss, g)
            dftfe_mlp_adam(self.params, g, m, v, t, lr)
            if t % 100 == 0 or t == 1:
                hist.append(float(loss.item()))
        return hist


class Controller:
    """Chooses the degree and bounds of each pass; `net` None = the standard rule only.

    With a network, at every potential change the network proposes the degree for the passes
    on that potential, the drift of theta_N for the first cut and the new upper bound (no
    Lanczos run); a = theta_N of the previous pass otherwise.  A proposed pass that does not
    halve the largest residual hands the rest of that potential to the standard rule."""

    def __init__(self, ham, nstates, net=None, seed=0):
        self.ham, self.N, self.net, self.seed = ham, nstates, net, seed
        self.hist = []
        self.b = None
        self.need_lanczos = True
        self.first_next = True
        self.learned_step = False
        self.step_m = FALLBACK_DEGREE
        self.step_a = None
        self.step_b = None
        self.lanczos_runs = 0
        self.fallbacks = 0
        self.proposed = 0

    def _lanczos_b(self):
        self.lanczos_runs += 1
        return dftfe_lanczos(self.ham, LANCZOS_K, seed=self.seed + 7919 * self.lanczos_runs)[2]

    def new_potential(self):
        self.first_next = True
        self.learned_step = False
        if self.net is not None and self.hist and self.b is not None:
            y = self.net.predict(features(self.hist, True))[0]
            if np.all(np.isfinite(y)):
                self.step_m, self.step_a, self.step_b, self.b = decode(y, self.hist[-1], self.b)
                self.learned_step = True
                self.proposed += 1
                return
        self.need_lanczos = True

    def propose(self):
        """(degree, bounds, mode) for the next pass."""
        if not self.hist:
            bd = dftfe_spectrum_bounds(self.ham, LANCZOS_K, self.seed, self.N)
            self.lanczos_runs += 1
            self.b = bd.b
            self.need_lanczos = False
            return FALLBACK_DEGREE, bd, "fallback"
        last = self.hist[-1]
        if self.learned_step:
            a = self.step_a if self.first_next else last.evals[-1]
            b = max(self.step_b, a + max(last.evals[-1] - last.evals[0], 1e-12))
            return self.step_m, make_bounds(a, b, last.evals[0]), "learned"
        if self.need_lanczos:
            self.b = self._lanczos_b()
            self.need_lanczos = False
        return FALLBACK_DEGREE, make_bounds(last.evals[-1], self.b, last.evals[0]), "fallback"

    def record(self, ev, rs, bounds, degree, mode):
        r = Record(ev.cpu().numpy(), rs.cpu().numpy(), bounds.a, bounds.b, degree, self.first_next)
        # progress is judged against the previous pass on the same potential only
        prev = self.hist[-1].rmax if self.hist and not self.first_next else math.inf
        self.hist = (self.hist + [r])[-3:]
        self.first_next = False
        if mode == "learned" and r.rmax > 0.5 * prev:
            self.learned_step = False          # the standard rule finishes this potential
            self.need_lanczos = True
            self.fallbacks += 1
        return r


_POTENTIALS = {}


def potentials(wl, qxyz, seed, steps, step_len=0.05, keep=0.3):
    """V_0 .. V_steps at the quadrature points: atoms walk `step_len` bohr per step and the
    potential is mixed keep * old + (1 - keep) * new (the SCF-like sequence).  The last
    sequence is kept, so the two controllers compared on it share one evaluation."""
    key = (wl.name, qxyz.shape, seed, steps, step_len, keep)
    if key in _POTENTIALS:
        return _POTENTIALS[key]
    _POTENTIALS.clear()
    _POTENTIALS[key] = V = _potentials(wl, qxyz, seed, steps, step_len, keep)
    return V


def _potentials(wl, qxyz, seed, steps, step_len, keep):
    import synth
    pts = qxyz.reshape(-1, 3)
    pos = synth.atom_walk(seed, wl.centres, steps, step_len)
    V = [synth.gaussian_wells(pts, pos[0], wl.depth, wl.width, wl.L)]
    for s in range(1, steps + 1):
        V.append(keep * V[-1] + (1.0 - keep) * synth.gaussian_wells(pts, pos[s], wl.depth, wl.width, wl.L))
    return V


def run_sequence(dg, ham, wl, qxyz, X, ctrl, seed, steps, tol=1e-5, max_passes=30, prec=0, search=False):
    """Converge every step of a potential sequence with `ctrl` (largest generalised residual of
    the lowest 3/4 of the states <= tol, see Judge); X (device, M x N) is the state carried
    from step to step.
    Returns per-step statistics and, with search=True, one training sample per potential
    change (from `search_step`, whose chosen degree then converges that step)."""
    import torch
    N = X.shape[1]
    nblk = (N + wl.block - 1) // wl.block
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    rs = torch.empty_like(ev)
    Vs = potentials(wl, qxyz, seed, steps)
    stats, samples = [], []
    judge = Judge()
    for s, V in enumerate(Vs):
        dg.dftfe_ham_set_potential(ham, torch.from_numpy(V).cuda())
        ctrl.new_potential()
        step_m = None
        if search and s > 0 and ctrl.hist:
            step_m, sample = search_step(ham, wl, X, ctrl, tol, prec, judge=judge)
            samples.append(sample)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        apps = passes = 0
        lz0 = ctrl.lanczos_runs
        while passes < max_passes:
            m, bd, mode = ctrl.propose()
            if step_m is not None:
                m = step_m
            dftfe_chfsi_pass(ham, X, wl.block, m, bd, ev, rs, prec)
            apps += m * nblk
            passes += 1
            ctrl.record(ev, rs, bd, m, mode)
            g = judge(ham, X, ev)
            if g <= tol:
                break
        torch.cuda.synchronize()
        stats.append(dict(step=s, passes=passes, applications=apps, lanczos=ctrl.lanczos_runs - lz0,
                          seconds=time.perf_counter() - t0, max_resid=g))
    return stats, samples


def run_batch_sequences(dg, systems, ctrls, steps, tol=1e-5, prec=2, max_passes=30):
    """Every system of `systems` (dicts with ham, wl, qxyz, X, seed, block) through its own
    SCF-like potential sequence, all systems together: at every step each system gets its new
    potential, then batched passes (dftfe_batch_chfsi_pass) run over the systems whose largest
    generalised residual of the lowest 3/4 of the states (Judge) is still above tol, each with
    the degree and bounds
    its controller proposes.  Returns per-step statistics (step 0 included)."""
    import torch
    n = len(systems)
    Vs = [potentials(sy["wl"], sy["qxyz"], sy["seed"], steps) for sy in systems]
    # the sequences of different systems are cached one at a time by potentials(): keep them here
    evs = [torch.empty(sy["X"].shape[1], dtype=torch.float64, device="cuda") for sy in systems]
    rss = [torch.empty_like(e) for e in evs]
    batches = {}
    stats = []
    judge = Judge()
    try:
        for st in range(steps + 1):
            for i, sy in enumerate(systems):
                dg.dftfe_ham_set_potential(sy["ham"], torch.from_numpy(Vs[i][st]).cuda())
                ctrls[i].new_potential()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            left = list(range(n))
            rounds = apps = 0
            lz0 = sum(c.lanczos_runs for c in ctrls)
            while left and rounds < max_passes:
                props = [ctrls[i].propose() for i in left]
                key = tuple(left)
                if key not in batches:
                    batches[key] = dg.dftfe_batch_create([systems[i]["ham"] for i in left])
                bds = [pr[1] for pr in props]
                dg.dftfe_batch_chfsi_pass(batches[key], [systems[i]["X"] for i in left],
                                          [systems[i]["block"] for i in left], [pr[0] for pr in props], bds,
                                          [evs[i] for i in left], [rss[i] for i in left], prec)
                rounds += 1
                still = []
                for j, i in enumerate(left):
                    m, _, mode = props[j]
                    N = systems[i]["X"].shape[1]
                    apps += m * ((N + systems[i]["block"] - 1) // systems[i]["block"])
                    ctrls[i].record(evs[i], rss[i], bds[j], m, mode)
                    if judge(systems[i]["ham"], systems[i]["X"], evs[i]) > tol:
                        still.append(i)
                left = still
            torch.cuda.synchronize()
            stats.append(dict(step=st, rounds=rounds, applications=apps, converged=not left,
                              lanczos=sum(c.lanczos_runs for c in ctrls) - lz0,
                              seconds=time.perf_counter() - t0))
    finally:
        for b in batches.values():
            dg.dftfe_batch_destroy(b)
    return stats


def search_step(ham, wl, X, ctrl, tol, prec, max_rollout=12, judge=None):
    """Targets at a potential change: from a copy of the state, each candidate degree is run
    with the standard bounds (fresh Lanczos bound, a = theta_N) until the tolerance is met,
    timed with the device synchronised on both sides; the target degree is the one with the
    least time to the tolerance (within 3 % of the least, the fewest filter applications).
    Returns it and the sample (features, targets)."""
    import torch
    last = ctrl.hist[-1]
    F = features(ctrl.hist, True)
    b_prev = last.b
    if ctrl.need_lanczos or ctrl.b is None:
        ctrl.b = ctrl._lanczos_b()
        ctrl.need_lanczos = False
    N = X.shape[1]
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    rs = torch.empty_like(ev)
    judge = judge or Judge()
    runs = {}
    nblk = (N + wl.block - 1) // wl.block
    for m in sorted(set(CANDIDATES) | {FALLBACK_DEGREE}):
        Xc = X.clone()
        a, a0 = last.evals[-1], last.evals[0]
        tn1 = None
        n = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(max_rollout):
            dftfe_chfsi_pass(ham, Xc, wl.block, m, make_bounds(a, ctrl.b, a0), ev, rs, prec)
            evh = ev.cpu().numpy()
            a, a0 = evh[-1], evh[0]
            if tn1 is None:
                tn1 = float(evh[-1])
            if judge(ham, Xc, ev) <= tol:
                n = k + 1
                break
        torch.cuda.synchronize()
        runs[m] = (n, tn1, time.perf_counter() - t0, (n or max_rollout) * m * nblk)
        del Xc
    done = {m: r for m, r in runs.items() if r[0] is not None}
    if not done:
        choice = FALLBACK_DEGREE
    else:
        best = min(r[2] for r in done.values())
        near = [m for m, r in done.items() if r[2] <= 1.03 * best]
        choice = min(near, key=lambda m: (done[m][3], m))
    spread = max(last.evals[-1] - last.evals[0], 1e-12)
    target = np.array([math.log2(choice / 16.0), (runs[choice][1] - last.evals[-1]) / spread,
                       math.log(ctrl.b / b_prev)])
    return choice, (F, target)


def _compare(dg, ham, wl, qxyz, start, net, seeds, steps, tol, prec, log):
    """Held-out sequences run twice from the same start: the standard rule and the proposer."""
    rows = []
    for s in seeds:
        row = {"seed": s}
        for name, n in (("standard", None), ("learned", net)):
            ctrl = Controller(ham, wl.nstates, n, s)
            stats, _ = run_sequence(dg, ham, wl, qxyz, start(s), ctrl, s, steps, tol, prec=prec)
            row[name] = {"applications": sum(x["applications"] for x in stats[1:]),
                         "passes": sum(x["passes"] for x in stats[1:]),
                         "seconds": sum(x["seconds"] for x in stats[1:]),
                         "lanczos_runs": ctrl.lanczos_runs, "fallbacks": ctrl.fallbacks,
                         "converged": all(x["max_resid"] <= tol for x in stats)}
        rows.append(row)
        log(row)
    tot = {}
    for k in ("applications", "passes", "seconds", "lanczos_runs"):
        tot[k] = {name: sum(r[name][k] for r in rows) for name in ("standard", "learned")}
    return rows, tot


def _system(dg, wl):
    import torch
    mesh = dg.dftfe_mesh_create(wl.L, wl.ncell, wl.degree)
    ham = dg.dftfe_ham_create(mesh)
    _, qxyz = dg.dftfe_mesh_coords(mesh, nodes=False)

    def start(seed):
        X = torch.empty((wl.ndofs, wl.nstates), dtype=torch.float64, device="cuda")
        dg.dftfe_random_uniform(X, 1000 + seed)
        return X
    return mesh, ham, qxyz, start


def experiment(train_seqs=24, test_seqs=5, steps=8, tol=1e-5, train_steps=3000, seed0=0, prec=0,
               eval_workload=None, eval_seqs=1, eval_steps=4, log=print):
    """Data from the degree search on `train_seqs` sequences of `steps` potentials of the
    13,824-DoF system (synth.small_wells: 8 wells, 32 states), training on the GPU kernels,
    then `test_seqs` held-out sequences of that system and, with `eval_workload` (a
    synth.Workload, e.g. the 32^3-cell, 1,024-state system), `eval_seqs` held-out sequences of
    `eval_steps` potentials of it, each run with the standard rule and with the proposer from
    the same start.  Passes in precision `prec`.  Returns a summary dictionary."""
    import paper_2203_07820_gb300 as dg
    import synth
    wl = synth.small_wells(seed0)
    mesh, ham, qxyz, start = _system(dg, wl)
    t0 = time.perf_counter()
    F, T = [], []
    for s in range(train_seqs):
        ctrl = Controller(ham, wl.nstates, None, s)
        _, samples = run_sequence(dg, ham, wl, qxyz, start(s), ctrl, s, steps, tol, prec=prec, search=True)
        F += [x[0] for x in samples]
        T += [x[1] for x in samples]
    t_data = time.perf_counter() - t0
    net = Network(seed=seed0 + 1)
    t0 = time.perf_counter()
    loss = net.train(np.array(F), np.array(T), steps=train_steps)
    t_train = time.perf_counter() - t0
    degrees = [int(round(16 * 2 ** t[0])) for t in T]
    out = {"system": wl.name, "ndofs": wl.ndofs, "nstates": wl.nstates, "tol": tol, "steps": steps,
           "precision": prec, "train_sequences": train_seqs, "samples": len(F),
           "target_degrees": {str(d): degrees.count(d) for d in sorted(set(degrees))},
           "data_seconds": t_data, "train_seconds": t_train, "loss_first_last": [loss[0], loss[-1]]}
    out["test"], out["test_total"] = _compare(dg, ham, wl, qxyz, start, net, range(1000, 1000 + test_seqs), steps,
                                              tol, prec, log)
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)
    if eval_workload is not None:
        wl2 = eval_workload
        mesh, ham, qxyz, start = _system(dg, wl2)
        rows, tot = _compare(dg, ham, wl2, qxyz, start, net, range(2000, 2000 + eval_seqs), eval_steps, tol, prec, log)
        out["eval"] = {"system": wl2.name, "ndofs": wl2.ndofs, "nstates": wl2.nstates, "steps": eval_steps,
                       "rows": rows, "total": tot}
        dg.dftfe_ham_destroy(ham)
        dg.dftfe_mesh_destroy(mesh)
    return out


if __name__ == "__main__":
    import argparse
    import json
    import synth
    ap = argparse.ArgumentParser(description="train and judge the learned degree/bounds proposer")
    ap.add_argument("--train-seqs", type=int, default=24)
    ap.add_argument("--test-seqs", type=int, default=5)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3"])
    ap.add_argument("--eval-scale32", action="store_true",
                    help="also evaluate on the 32^3-cell, p = 6, 1,024-state system (7,077,888 DoFs)")
    ap.add_argument("--eval-seqs", type=int, default=1)
    ap.add_argument("--eval-steps", type=int, default=4)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    prec = {"fp64": 0, "tf32x3": 2}[a.precision]
    ev = synth.lattice_atoms(0, ncell=32, nstates=1024, passes=2) if a.eval_scale32 else None
    res = experiment(a.train_seqs, a.test_seqs, a.steps, prec=prec, eval_workload=ev, eval_seqs=a.eval_seqs,
                     eval_steps=a.eval_steps)
    print(json.dumps({k: v for k, v in res.items() if k != "test"}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
