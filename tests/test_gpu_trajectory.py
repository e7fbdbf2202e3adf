"""Per-replication trajectories of the GPU pairs against the CPU oracle (needs a GB300).

The recording variant of the sampling kernel (params.trace_steps) writes, for the first
replications of every traced slot, the meeting time tau (Theorem 1(d): the first t >= L with
X_t = Y_{t-L}), the completion time C = max(l, tau) of Algorithm 3, and per draw t the site I_t and
which chains that draw moved (X_{t+1}, and from t = L on Y_{t+1-L}).  The oracle computes each
replication on its own from its stored paths (oracle.Model.replication).  Everything is compared
element by element: the same sites, the same flips, the same tau and C, in the kernel build the
run would use (compile-time degree, mask-indexed thresholds, the meeting-cap and lag variant), and
the recording variant gives the same integer sums as the production one."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_30239_gb300 import build, mcpd
    build.build()
    c = mcpd.Context(0)
    yield c
    c.close()


def _run(ctx, inst, **kw):
    import torch
    from paper_2608_30239_gb300 import mcpd
    plan = mcpd.Plan(ctx, inst, **kw)
    est = torch.empty(plan.n_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    plan.run_async(est, se)
    st = plan.collect()
    out = dict(stats=st, est=est.cpu().numpy(), se=se.cpu().numpy(), **plan.buckets())
    if kw.get("trace_steps"):
        out["rec"] = plan.fetch(mcpd.MCPD_FETCH_TRACE_REC)
        out["reps"] = plan.fetch(mcpd.MCPD_FETCH_SLOT_REPS)
    plan.close()
    return out


def _check_slot(M, run, rec_slot, p, reps, lag, steps):
    """rec_slot: [trace_reps][4 + steps] records of slot p, which started `reps` replications."""
    checked = 0
    for r in range(rec_slot.shape[0]):
        rec = rec_slot[r]
        if r >= reps:
            assert not rec.any(), (p, r)                  # never started: untouched
            continue
        status, C_gpu = int(rec[2]), int(rec[1])
        assert status in (1, 2) and int(rec[3]) == r, (p, r, status)
        C = M.replication(run, p, r)["C"]                   # size the stored paths to the replication
        o = M.replication(run, p, r, traj_cap=C + 1)
        assert o["status"] == 0 and o["C"] == C
        if status == 1:                                   # completed: same tau and C
            assert (int(rec[0]), C_gpu) == (o["tau"], o["C"]), (p, r)
        else:                                             # stopped as doomed before completing
            assert C_gpu <= o["C"] and int(rec[0]) in (0, o["tau"]), (p, r)
        X, Y, sites = o["X"].astype(np.int64), o["Y"].astype(np.int64), o["sites"]
        n = min(C_gpu, steps)
        words = rec[4:4 + n].astype(np.int64)
        assert np.array_equal(words & 0xFFFF, sites[:n]), (p, r)
        xf = (X[1:n + 1] != X[:n]).any(axis=1)
        yf = np.zeros(n, bool)
        if n > lag:
            yf[lag:] = (Y[1:n + 1 - lag] != Y[:n - lag]).any(axis=1)
        assert np.array_equal((words >> 16) & 1, xf.astype(np.int64)), (p, r)
        assert np.array_equal((words >> 17) & 1, yf.astype(np.int64)), (p, r)
        assert not rec[4 + n:].any()
        checked += 1
    return checked


CASES = {
    # tiny design with refill: several replications per slot, the last often stopped as doomed
    "tiny-refill": (lambda: synth.tiny_config(1), dict(slots=700, k=3, ell=20, horizon=60, seed=31), None),
    # degree 6 (compile-time degree, mask-indexed thresholds), the high-noise rates
    "degree6-high-noise": (lambda: synth.make_instance(300, 30, 6, 3, 0.10, 0.20, 3 / 300, 71, 72),
                           dict(slots=1500, k=31, ell=300, horizon=900, seed=811), None),
    # mixed degrees (generic build), random start, lag 3 and a meeting cap (the EXT variant)
    "mixed-lag-cap": (lambda: synth.make_mixed_instance(150, 14, 2, 6, 2, 0.05, 0.15, 2 / 150, 91, 92),
                      dict(slots=900, k=16, ell=150, horizon=600, seed=5, lag=3, meeting_cap=300),
                      "random"),
    # the largest instances of the batched workload (n = 5000, m = 385, 8 pools per clone)
    "n5000-degree8": (lambda: synth.make_instance(5000, 385, 8, 4, 0.05, 0.15, 4 / 5000, 41, 42),
                      dict(slots=300, k=501, ell=5000, horizon=10000, seed=12), None),
    # the uncoupled comparators (Algorithms 1 and 2): one chain, sites and flips of X only
    "uncoupled-systematic": (lambda: synth.make_instance(200, 20, 4, 2, 0.05, 0.1, 2 / 200, 51, 52),
                             dict(slots=700, coupled=False, scan=2, burn=20, length=180, horizon=700,
                                  seed=21), None),
    "uncoupled-score-degree6": (lambda: synth.make_instance(300, 30, 6, 3, 0.10, 0.20, 3 / 300, 71, 72),
                                dict(slots=700, coupled=False, burn=30, length=270, horizon=900, seed=22),
                                "random"),
    # a Tapestry-shaped regular design (961 x 93, 3 pools per sample, 31 samples per pool)
    "tapestry-961": (lambda: synth.make_tapestry_like_instance(961, 93, 3, 3, 0.05, 0.10, 3 / 961, 43, 44),
                     dict(slots=800, k=97, ell=961, horizon=2000, seed=13), "random"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_trajectories_match_the_oracle(ctx, case):
    make, kw, start = CASES[case]
    inst = make()
    nu = np.random.default_rng(9).uniform(0.0, 0.25, inst.n) if start == "random" else None
    steps, reps, stride = 512, 6, 7
    g = _run(ctx, inst, init_marginals=nu, record_slots=True, trace_stride=stride, trace_steps=steps,
             trace_reps=reps, **kw)
    plain = _run(ctx, inst, init_marginals=nu, **kw)
    for key in ("S1", "S2_lo", "S2_hi", "count"):          # recording changes no result
        assert np.array_equal(g[key], plain[key]), key
    assert np.array_equal(g["est"], plain["est"])
    if kw.get("coupled", True):
        M = oracle.Model(inst, init_marginals=nu)
        run = oracle.coupled_run(kw["k"], kw["ell"], kw["horizon"], kw["seed"],
                                 meeting_cap=kw.get("meeting_cap", 0), lag=kw.get("lag", 1))
    else:
        M = oracle.Model(inst, init_marginals=nu,
                         scan=oracle.SCAN_SYSTEMATIC if kw.get("scan") == 2 else oracle.SCAN_SCORE)
        run = oracle.uncoupled_run(kw["burn"], kw["length"], kw["horizon"], kw["seed"])
    checked = 0
    for idx, p in enumerate(range(0, kw["slots"], stride)):
        checked += _check_slot(M, run, g["rec"][idx], p, int(g["reps"][p]), kw.get("lag", 1), steps)
    assert checked >= min(100, kw["slots"] // stride)


def test_full_size_trajectories(ctx):
    """The bench's workload (1298 x 97 high noise, 524288 slots, budget 4e10) in its launch shape:
    13 slots spread over the run, their first four replications, 4096 draws each."""
    inst = synth.high_noise_config()
    P, stride, steps = 524288, 524288 // 12 + 1, 4096
    g = _run(ctx, inst, slots=P, budget_site_updates=4e10, seed=20260, record_slots=True,
             trace_stride=stride, trace_steps=steps, trace_reps=4)
    M = oracle.Model(inst)
    k, ell = oracle.window_defaults(inst.n, 1)
    run = oracle.coupled_run(k, ell, synth.budget_horizon(4e10, P), 20260)
    checked = 0
    for idx, p in enumerate(range(0, P, stride)):
        checked += _check_slot(M, run, g["rec"][idx], p, int(g["reps"][p]), 1, steps)
    assert checked >= 13 * 3
