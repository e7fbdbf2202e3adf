"""GPU path vs the CPU oracle, through the C ABI (needs a GB300).

Integer outputs (N*_p buckets of sum G and sum G^2, per-slot N*_p, retained cost, replication
counts, traced G vectors) must be bit-exact; the finalized doubles too, since both sides evaluate
the same correctly rounded expression on the same integers (the bound north of that is 1e-12
relative, asserted as equality here)."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


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


def _gpu_run(ctx, inst, **kw):
    import torch
    from paper_2608_30239_gb300 import mcpd
    plan = mcpd.Plan(ctx, inst, **kw)
    est = torch.empty(plan.n_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    plan.run_async(est, se)
    stats = plan.collect(allow_step_limit=True)
    out = dict(plan=plan, est=est.cpu().numpy(), se=se.cpu().numpy(), stats=stats)
    out.update(plan.buckets())
    if kw.get("record_slots"):
        out["slot_nstar"] = plan.fetch(mcpd.MCPD_FETCH_SLOT_NSTAR)
        out["slot_S"] = plan.fetch(mcpd.MCPD_FETCH_SLOT_S)
        out["slot_reps"] = plan.fetch(mcpd.MCPD_FETCH_SLOT_REPS)
    if kw.get("trace_stride"):
        out["trace_G"] = plan.fetch(mcpd.MCPD_FETCH_TRACE_G)
    return out


def _oracle_run(inst, P, k, ell, B, seed, coupled=True, burn=0, length=1, n_active=0,
                scan=oracle.SCAN_SCORE, custom_w=None, init=None, slot_offset=0, slot_G=False,
                meeting_cap=0, lag=1):
    M = oracle.Model(inst, n_active=n_active, scan=scan, custom_w=custom_w, init_marginals=init)
    run = (oracle.coupled_run(k, ell, B, seed, slot_offset=slot_offset, meeting_cap=meeting_cap, lag=lag) if coupled
           else oracle.uncoupled_run(burn, length, B, seed, slot_offset=slot_offset))
    res = M.run_slots(run, 0, P, THREADS, per_slot=True, slot_G=slot_G)
    L = (ell - k + 1) if coupled else length
    res["est"], res["se"] = M.finalize(res, P, L)
    return res


def _assert_same(g, o, per_slot=True):
    for key in ("S1", "S2_lo", "S2_hi", "count"):
        assert np.array_equal(g[key], o[key]), key
    if per_slot:
        assert np.array_equal(g["slot_nstar"], o["slot_nstar"])
        assert np.array_equal(g["slot_S"], o["slot_S"])
    assert np.array_equal(g["est"], o["est"])
    assert np.array_equal(g["se"], o["se"], equal_nan=True)


def test_device_philox_matches_oracle(ctx):
    import torch
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    d_ctr = torch.from_numpy(ctr.view(np.int32).copy()).cuda()
    d_out = torch.empty_like(d_ctr)
    key = (0xA4093822, 0x299F31D0)
    ctx.philox(d_ctr, key[0], key[1], d_out, len(ctr))
    got = d_out.cpu().numpy().view(np.uint32)
    for i in range(0, len(ctr), 97):
        assert np.array_equal(got[i], oracle.philox(ctr[i], key))


@pytest.mark.parametrize("k,ell", [(3, 20), (0, 0), (0, 1), (20, 20)])
def test_tiny_one_replication_per_slot(ctx, k, ell):
    """20 clones x 8 pools, 4096 pairs run to meeting (B = 0: every slot keeps its first pair)."""
    inst = synth.tiny_config(1)
    P = 4096
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=0, seed=77, record_slots=True)
    o = _oracle_run(inst, P, k, ell, 0, 77)
    _assert_same(g, o)
    assert g["stats"]["reps_started"] == P and g["stats"]["zero_completion_slots"] == P


@pytest.mark.parametrize("B", [0, 25, 60, 400])
def test_tiny_refill(ctx, B):
    inst = synth.tiny_config(2)
    P = 3001
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=B, seed=5, record_slots=True,
                 trace_stride=1)
    o = _oracle_run(inst, P, 3, 20, B, 5, slot_G=True)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"])


def test_medium_design_refill_ragged(ctx):
    """400 clones x 31 pools (k = 5): several blocks, a ragged last wave, per-slot G vectors."""
    inst = synth.make_instance(400, 31, 5, 3, 0.05, 0.1, 3 / 400, 41, 42)
    P = 7777
    k, ell = oracle.window_defaults(400, 1)
    B = 5 * ell + 17
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=2024, record_slots=True,
                 trace_stride=7)
    o = _oracle_run(inst, P, k, ell, B, 2024, slot_G=True)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"][::7])


def test_bernoulli_initial_state(ctx):
    inst = synth.tiny_config(3)
    rng = np.random.default_rng(3)
    nu = rng.random(inst.n)
    nu[0], nu[1], nu[2] = 0.0, 1.0, 0.5
    P = 2000
    g = _gpu_run(ctx, inst, slots=P, k=2, ell=15, horizon=70, seed=9, init_marginals=nu,
                 record_slots=True)
    o = _oracle_run(inst, P, 2, 15, 70, 9, init=nu)
    _assert_same(g, o)


@pytest.mark.parametrize("scan", ["score", "uniform", "systematic"])
def test_uncoupled_comparators(ctx, scan):
    from paper_2608_30239_gb300 import mcpd
    inst = synth.make_instance(120, 12, 4, 2, 0.05, 0.1, 2 / 120, 7, 8)
    code = {"score": 0, "uniform": 1, "systematic": 2}[scan]
    P = 1500
    g = _gpu_run(ctx, inst, slots=P, coupled=False, scan=code, burn=12, length=108, horizon=600,
                 seed=31, record_slots=True)
    o = _oracle_run(inst, P, 0, 0, 600, 31, coupled=False, burn=12, length=108, scan=code)
    _assert_same(g, o)
    assert g["stats"]["site_updates"] == P * (600 // 119) * 119
    _ = mcpd


@pytest.mark.parametrize("scan,deg", [("score", 6), ("systematic", 6), ("uniform", 5), ("systematic", 3)])
def test_uncoupled_degree_builds(ctx, scan, deg):
    """Uncoupled comparators on uniform-degree designs (the builds compiled for the degree, with
    mask-indexed thresholds), including the high-noise shape at degree 6."""
    inst = synth.make_instance(300, 30, deg, 3, 0.10, 0.20, 3 / 300, 60 + deg, 61 + deg)
    code = {"score": 0, "uniform": 1, "systematic": 2}[scan]
    P, burn, length = 2000, 30, 270
    g = _gpu_run(ctx, inst, slots=P, coupled=False, scan=code, burn=burn, length=length, horizon=900,
                 seed=41 + deg, record_slots=True)
    o = _oracle_run(inst, P, 0, 0, 900, 41 + deg, coupled=False, burn=burn, length=length, scan=code)
    _assert_same(g, o)


def test_custom_weights_and_pruning(ctx):
    inst = synth.high_noise_config()
    P = 600
    na = 333
    w = np.linspace(1.0, 3.0, na)
    k, ell = oracle.window_defaults(na, 1)
    g = _gpu_run(ctx, inst, slots=P, n_active=na, scan=3, scan_weights=w, k=k, ell=ell,
                 horizon=3 * ell, seed=4, record_slots=True)
    o = _oracle_run(inst, P, k, ell, 3 * ell, 4, n_active=na, scan=oracle.SCAN_CUSTOM, custom_w=w)
    _assert_same(g, o)


def test_decode_host_api_matches_plan(ctx):
    """mcpd_decode (host arrays, original clone order, pruned clones 0) equals the plan path."""
    inst = synth.high_noise_config()
    kw = dict(slots=512, n_active=333, horizon=2000, seed=11)
    d = ctx.decode(inst, **kw)
    g = _gpu_run(ctx, inst, **kw)
    act = g["plan"].active
    assert np.array_equal(np.flatnonzero(d["active"]), act)
    assert np.array_equal(d["est"][act], g["est"])
    assert np.array_equal(d["se"][act], g["se"])
    pruned = np.setdiff1d(np.arange(inst.n), act)
    assert np.all(d["est"][pruned] == 0) and np.all(d["se"][pruned] == 0)


@pytest.mark.parametrize("audit", [1, 5, 40])
def test_tau_audit_counts_meetings_beyond_the_threshold(ctx, audit):
    """With one replication per slot (B = 0), the audit count equals the number of slots whose
    oracle replication met at tau > audit, and the sums are those of an unaudited run."""
    inst = synth.tiny_config(4)
    P = 4096
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=0, seed=55, tau_audit=audit)
    M = oracle.Model(inst)
    run = oracle.coupled_run(3, 20, 0, 55)
    taus = np.array([M.replication(run, p)["tau"] for p in range(P)])
    assert g["stats"]["tau_over_audit"] == int((taus > audit).sum())
    assert g["stats"]["max_tau"] == int(taus.max()) and g["stats"]["sum_tau"] == int(taus.sum())
    plain = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=0, seed=55)
    assert np.array_equal(plain["S1"], g["S1"]) and plain["stats"]["tau_over_audit"] == 0


def test_tau_audit_with_refill(ctx):
    """With refill (B = 60, several replications per slot and many slots per pair), the audit
    count equals the number of retained oracle replications that met at tau > audit, and the
    retained count is unchanged by the audit."""
    inst = synth.tiny_config(4)
    P, audit = 1500, 3
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=60, seed=56, tau_audit=audit)
    M = oracle.Model(inst)
    run = oracle.coupled_run(3, 20, 60, 56)
    res = M.run_slots(run, 0, P, per_slot=True)
    taus = np.array([M.replication(run, p, r)["tau"] for p in range(P) for r in range(int(res["slot_nstar"][p]))])
    assert g["stats"]["reps_retained"] == taus.size == int(res["slot_nstar"].sum())
    assert g["stats"]["tau_over_audit"] == int((taus > audit).sum()) > 0
    assert g["stats"]["sum_tau"] == int(taus.sum())


@pytest.mark.parametrize("cap,B", [(20, 0), (24, 0), (20, 60), (24, 60), (90, 400)])
def test_meeting_cap(ctx, cap, B):
    """The finite meeting cap: a pair unmet at t = cap is kept with every inner sum cut at the
    cap.  Bit-exact against the oracle with the same cap, with and without refill; the audit,
    which defaults to the cap, counts the capped pairs that were kept.  (20, 60): every
    replication costs exactly 20, so the third one of a slot reaches the cap at the very clock
    B - S at which an unfinished replication is doomed; capped, it is kept."""
    inst = synth.tiny_config(4)
    P = 3001
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=B, seed=57, meeting_cap=cap,
                 record_slots=True, trace_stride=1)
    o = _oracle_run(inst, P, 3, 20, B, 57, meeting_cap=cap, slot_G=True)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"])
    assert g["stats"]["step_limit_hits"] == 0
    if B == 0:                 # every replication is kept: the counts agree exactly
        assert g["stats"]["tau_over_audit"] == o["stats"]["capped"] > 0
        assert g["stats"]["sum_tau"] == o["stats"]["sum_tau"]
    else:                      # the oracle also counts the discarded last replication of a slot
        assert 0 < g["stats"]["tau_over_audit"] <= o["stats"]["capped"]


def test_meeting_cap_mixed_degree_random_start(ctx):
    """The cap on a mixed-degree design (padding pools) from a random start, where Y_0 carries
    bits that no flip of the replication touched."""
    inst = _mixed()
    nu = np.random.default_rng(8).random(inst.n) * 0.2
    k, ell = oracle.window_defaults(inst.n, 1)
    P, B, cap = 3000, 3 * ell + 5, ell + 9
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=809, init_marginals=nu,
                 meeting_cap=cap, record_slots=True, trace_stride=7)
    o = _oracle_run(inst, P, k, ell, B, 809, init=nu, slot_G=True, meeting_cap=cap)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"][::7])
    assert g["stats"]["tau_over_audit"] > 0


@pytest.mark.parametrize("lag,B,cap", [(2, 0, 0), (2, 60, 0), (5, 400, 0), (5, 90, 30), (25, 200, 0)])
def test_lag_coupling(ctx, lag, B, cap):
    """Lag-L pairs (L pre-lag updates of X, then X_{t+1} and Y_{t+1-L} from the same draw),
    with and without refill and a meeting cap: bit-exact against the oracle; the site updates
    count L pre-lag updates per replication."""
    inst = synth.tiny_config(4)
    P = 3001
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=B, seed=58, lag=lag, meeting_cap=cap,
                 record_slots=True, trace_stride=1)
    o = _oracle_run(inst, P, 3, 20, B, 58, lag=lag, meeting_cap=cap, slot_G=True)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"])
    st = g["stats"]
    assert st["step_limit_hits"] == 0
    assert st["site_updates"] == 2 * st["progress_units"] - lag * st["reps_started"]
    if B == 0:
        assert st["progress_units"] == o["stats"]["draws"] and st["sum_tau"] == o["stats"]["sum_tau"]
        assert st["max_tau"] >= lag


@pytest.mark.parametrize("lag", [3, 12])
def test_lag_random_start_mixed_degree(ctx, lag):
    """Lag on a mixed-degree design from a random start: Y_0 is copied at the first pre-lag move,
    X may come back to Y_0 before t = L (the meeting is then decided at t = L)."""
    inst = _mixed()
    nu = np.random.default_rng(9).random(inst.n) * 0.2
    k, ell = 5, 40
    P, B = 3000, 300
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=810, init_marginals=nu, lag=lag,
                 record_slots=True, trace_stride=5)
    o = _oracle_run(inst, P, k, ell, B, 810, init=nu, slot_G=True, lag=lag)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"][::5])


def test_lag_degree_six(ctx):
    """The degree-6 kernel (mask-indexed thresholds) with lag 4 and the high-noise shape."""
    inst = synth.make_instance(300, 30, 6, 3, 0.10, 0.20, 3 / 300, 71, 72)
    k, ell = oracle.window_defaults(inst.n, 1)
    P, B = 2000, 3 * ell
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=811, lag=4, record_slots=True)
    o = _oracle_run(inst, P, k, ell, B, 811, lag=4)
    _assert_same(g, o)


@pytest.mark.parametrize("case", ["one_slot", "all_negative", "all_positive", "one_active"])
def test_degenerate_inputs(ctx, case):
    """Edge cases: a single slot (its standard error is undefined, NaN on both sides), every pool
    negative, every pool positive, and pruning to a single active clone; bit-exact against the
    oracle."""
    import dataclasses
    inst = synth.tiny_config(3)
    P, B, n_active = 777, 90, 0
    if case == "one_slot":
        P = 1
    elif case == "all_negative":
        inst = dataclasses.replace(inst, y=np.zeros_like(inst.y))
    elif case == "all_positive":
        inst = dataclasses.replace(inst, y=np.ones_like(inst.y))
    else:
        n_active = 1
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=B, seed=61, n_active=n_active, record_slots=True)
    o = _oracle_run(inst, P, 3, 20, B, 61, n_active=n_active)
    _assert_same(g, o)
    if case == "one_slot":
        assert np.all(np.isnan(g["se"])) and np.all(np.isfinite(g["est"]))
    if case == "one_active":
        assert g["est"].shape == (1,)


@pytest.mark.parametrize("variant", ["plain", "random_start", "cap_lag_random_start"])
@pytest.mark.parametrize("P", [1, 2, 5, 33, 97])
def test_few_live_lanes_per_warp(ctx, variant, P):
    """Far fewer slots than the launch has threads, so most warps hold one or a few lanes with
    work, and lanes leave while others go on. The ends of replications and the random starts
    that the live lanes of a warp share (split by rank among them) must still cover every word
    of the ending lane's column. Refill on a 300-clone design (10 bit words per column), plain,
    from a random start, and from a random start with lag 3 and a meeting cap; bit-exact
    against the oracle, per slot and in every slot's G record."""
    inst = synth.make_instance(300, 24, 5, 3, 0.05, 0.15, 3 / 300, 501, 502)
    k, ell, B, seed = 31, 300, 1200, 4242
    kw, okw = {}, {}
    if variant != "plain":
        nu = np.random.default_rng(12).random(inst.n) * 0.2
        kw["init_marginals"] = nu
        okw["init"] = nu
    if variant == "cap_lag_random_start":
        kw.update(meeting_cap=2 * ell, lag=3)
        okw.update(meeting_cap=2 * ell, lag=3)
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=seed, record_slots=True,
                 trace_stride=1, **kw)
    o = _oracle_run(inst, P, k, ell, B, seed, slot_G=True, **okw)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"])


def test_near_maximum_pair_state(ctx):
    """6560 clones x 200 pools, 4 pools per clone: a chain's column is 256 words, the most that
    15-bit count offsets address, and the staged tables (161 KB) with one warp region and one Y
    region fill 221 KB of shared memory, so the launch runs one warp per block; bit-exact against
    the oracle with refill."""
    inst = synth.make_instance(6560, 200, 4, 5, 0.10, 0.20, 5 / 6560, 4401, 4402)
    P, B = 96, 600
    g = _gpu_run(ctx, inst, slots=P, k=20, ell=200, horizon=B, seed=71, record_slots=True)
    o = _oracle_run(inst, P, 20, 200, B, 71)
    _assert_same(g, o)
    assert int(g["plan"].info[7]) == 1                  # warps per block


def test_pair_state_too_large_is_refused(ctx):
    """A design whose pair state is beyond 15-bit count offsets (60000 clones) is refused when the
    plan is made (MCPD_ETOO_LARGE); the context still decodes afterwards."""
    from paper_2608_30239_gb300 import mcpd
    big = synth.make_instance(60000, 1022, 3, 5, 0.05, 0.10, 5 / 60000, 4403, 4404)
    with pytest.raises(mcpd.McpdError) as ei:
        mcpd.Plan(ctx, big, slots=64, k=20, ell=200, horizon=0, seed=1)
    assert ei.value.code == mcpd.MCPD_ETOO_LARGE
    inst = synth.tiny_config(2)
    g = _gpu_run(ctx, inst, slots=256, k=3, ell=20, horizon=0, seed=5)
    o = _oracle_run(inst, 256, 3, 20, 0, 5)
    _assert_same(g, o, per_slot=False)


def test_step_limit_reports_error_and_context_survives(ctx):
    from paper_2608_30239_gb300 import mcpd
    inst = synth.tiny_config(1)
    g = _gpu_run(ctx, inst, slots=256, k=3, ell=20, horizon=0, seed=77, step_limit=25)
    assert g["stats"]["status"] == mcpd.MCPD_ESTEP_LIMIT
    assert g["stats"]["step_limit_hits"] > 0
    again = _gpu_run(ctx, inst, slots=256, k=3, ell=20, horizon=0, seed=77)
    assert again["stats"]["status"] == mcpd.MCPD_OK


@pytest.mark.parametrize("deg", [4, 7, 8])
def test_uniform_degree_variants(ctx, deg):
    """Kernels compiled for a uniform degree: 4 (mask-indexed thresholds), 7 and 8 (coded
    thresholds); coupled with refill, against the oracle."""
    inst = synth.make_instance(230, 21, deg, 4, 0.08, 0.15, 4 / 230, 70 + deg, 80 + deg)
    k, ell = oracle.window_defaults(inst.n, 1)
    P, B = 2500, 3 * ell + 11
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=313, record_slots=True)
    o = _oracle_run(inst, P, k, ell, B, 313)
    _assert_same(g, o)


@pytest.mark.parametrize("n,m", [(320, 48), (961, 93)])
def test_tapestry_shaped_designs(ctx, n, m):
    """The shapes of the paper's Tapestry designs (each sample in 3 pools; 320 x 48 and 961 x 93),
    drawn as regular designs: coupled score-weighted decoding with refill equals the oracle."""
    inst = synth.make_tapestry_like_instance(n, m, 3, 3, 0.05, 0.10, 3 / n, 90 + m, 91 + m)
    k, ell = oracle.window_defaults(inst.n, 1)
    P, B = 2000, 5 * ell
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=420, record_slots=True)
    o = _oracle_run(inst, P, k, ell, B, 420)
    _assert_same(g, o)


def _mixed():
    """260 clones x 23 pools, each clone in 2 to 8 pools: rows padded to the longest."""
    return synth.make_mixed_instance(260, 23, 2, 8, 6, 0.1, 0.2, 6 / 260, 31, 32)


@pytest.mark.parametrize("start", ["all_negative", "bernoulli"])
def test_mixed_degree_design(ctx, start):
    """Clones in different numbers of pools (the padding entries must never count as deciding
    pools, in either chain), coupled with refill; the random start copies Y_0 after a pre-lag
    flip."""
    inst = _mixed()
    nu = None
    if start == "bernoulli":
        nu = np.random.default_rng(5).random(inst.n) * 0.2
    k, ell = oracle.window_defaults(inst.n, 1)
    P, B = 3000, 3 * ell + 5
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=808, init_marginals=nu,
                 record_slots=True, trace_stride=11)
    o = _oracle_run(inst, P, k, ell, B, 808, init=nu, slot_G=True)
    _assert_same(g, o)
    assert np.array_equal(g["trace_G"], o["slot_G"][::11])
    assert g["stats"]["sum_tau"] > g["stats"]["reps_retained"]     # unmet stretches did occur


def test_mixed_degree_uncoupled(ctx):
    inst = _mixed()
    P = 1200
    g = _gpu_run(ctx, inst, slots=P, coupled=False, burn=20, length=240, horizon=900, seed=6,
                 record_slots=True)
    o = _oracle_run(inst, P, 0, 0, 900, 6, coupled=False, burn=20, length=240)
    _assert_same(g, o)


def test_unmet_pairs_overflow_shared_y(ctx):
    """An instance whose pairs stay unmet about half of the time (200 x 20, k = 3, 8 positives,
    fp .2, fn .3): far more pairs are unmet at once than the shared Y regions hold, so many use
    their global Y column.  Sampled slots equal the oracle's, and every slot is accounted for."""
    inst = synth.make_instance(200, 20, 3, 8, 0.2, 0.3, 8 / 200, 11, 12)
    k, ell = oracle.window_defaults(inst.n, 1)
    P, B, stride = 120_000, 2 * ell, 1499
    g = _gpu_run(ctx, inst, slots=P, k=k, ell=ell, horizon=B, seed=99, record_slots=True,
                 trace_stride=stride)
    st = g["stats"]
    assert st["status"] == 0 and int(g["count"].sum()) == P
    assert st["sum_tau"] > 0.3 * st["progress_units"]
    M = oracle.Model(inst)
    for idx, p in enumerate(range(0, P, stride)):
        run = oracle.coupled_run(k, ell, B, 99, slot_offset=p)
        r = M.run_slots(run, 0, 1, 1, per_slot=True, slot_G=True)
        assert g["slot_nstar"][p] == r["slot_nstar"][0]
        assert g["slot_S"][p] == r["slot_S"][0]
        assert np.array_equal(g["trace_G"][idx], r["slot_G"][0]), p


# -------------------------------------------------------------------------------------------
# Full size: the 1298 x 97 high-noise configuration with 524288 slots and a 4e10 site-update
# budget, in the launch configuration the bench times.  Sampled slots are recomputed one by one.
P_FULL = 524288
BUDGET = 4e10


@pytest.fixture(scope="module")
def full_run(ctx):
    inst = synth.high_noise_config()
    stride = P_FULL // 12 + 1
    g = _gpu_run(ctx, inst, slots=P_FULL, budget_site_updates=BUDGET, seed=20260,
                 record_slots=True, trace_stride=stride)
    return inst, stride, g


def test_full_size_sampled_slots_bit_exact(full_run):
    inst, stride, g = full_run
    M = oracle.Model(inst)
    k, ell = oracle.window_defaults(inst.n, 1)
    B = synth.budget_horizon(BUDGET, P_FULL)
    for idx, p in enumerate(range(0, P_FULL, stride)):
        run = oracle.coupled_run(k, ell, B, 20260, slot_offset=p)
        r = M.run_slots(run, 0, 1, 1, per_slot=True, slot_G=True)
        assert g["slot_nstar"][p] == r["slot_nstar"][0]
        assert g["slot_S"][p] == r["slot_S"][0]
        assert np.array_equal(g["trace_G"][idx], r["slot_G"][0]), p


def test_full_size_properties(full_run):
    inst, stride, g = full_run
    st = g["stats"]
    assert st["status"] == 0
    assert int(g["count"].sum()) == P_FULL
    assert np.array_equal(np.bincount(g["slot_nstar"], minlength=len(g["count"]) + 1)[1:], g["count"])
    assert st["site_updates"] <= 2 * st["progress_units"]
    assert np.all(np.isfinite(g["est"])) and np.all(g["se"] >= 0)
    # a clone that never turned positive in any chain has G = 0 in every slot: estimate 0, se 0
    assert np.all(g["est"][g["se"] == 0] == 0)
    # the bucketed integer sums reproduce the per-slot bookkeeping
    B = synth.budget_horizon(BUDGET, P_FULL)
    assert np.all(g["slot_S"][g["slot_nstar"] > 1] <= B)
    assert st["reps_retained"] == int(g["slot_nstar"].sum())


def test_full_size_partition_and_determinism(ctx, full_run):
    """Two launches over slot halves (global ids via slot_offset) sum to the one-launch buckets, and
    a rerun is bit-identical: integer sums do not depend on the schedule."""
    inst, stride, g = full_run
    half = P_FULL // 2
    a = _gpu_run(ctx, inst, slots=half, horizon=synth.budget_horizon(BUDGET, P_FULL), seed=20260)
    b = _gpu_run(ctx, inst, slots=half, horizon=synth.budget_horizon(BUDGET, P_FULL), seed=20260,
                 slot_offset=half)
    assert np.array_equal(a["S1"] + b["S1"], g["S1"])
    lo = a["S2_lo"] + b["S2_lo"]
    carry = (lo < a["S2_lo"]).astype(np.uint64)
    assert np.array_equal(lo, g["S2_lo"])
    assert np.array_equal(a["S2_hi"] + b["S2_hi"] + carry, g["S2_hi"])
    again = _gpu_run(ctx, inst, slots=P_FULL, budget_site_updates=BUDGET, seed=20260)
    assert np.array_equal(again["S1"], g["S1"])
    assert np.array_equal(again["est"], g["est"])


# -------------------------------------------------------------------------------------------
# The other workload configurations at their full sizes.
def test_tiny_workload_against_the_exact_posterior(ctx):
    """The tiny workload (20 clones x 8 pools, 3 pools per clone, 2 positives, fp .02, fn .05,
    q .01; 4096 lag-1 pairs with the paper's score weights, each run to meeting, k = 3, l = 20):
    bit-exact with the oracle, and within sampling error of the exact posterior marginals of the
    2^20 enumeration (z < 4.5 for every clone)."""
    from oracle import exact
    inst = synth.tiny_config(1)
    P = 4096
    g = _gpu_run(ctx, inst, slots=P, k=3, ell=20, horizon=0, seed=2026, record_slots=True)
    o = _oracle_run(inst, P, 3, 20, 0, 2026)
    _assert_same(g, o)
    _, p = exact.posterior(inst)
    z = np.abs(g["est"] - p) / np.where(g["se"] > 0, g["se"], np.inf)
    assert np.all(z < 4.5), z
    assert np.all(g["est"][g["se"] == 0] == 0.0)        # a clone never positive in any chain


@pytest.mark.parametrize("method", ["coupled-score", "uncoupled-systematic"])
def test_library_workload_full_size_sampled_slots(ctx, method):
    """The paper-shaped library workload (1298 x 97, 6 pools per clone, 3 positives, fp .01, fn .05,
    q = 3/1298) at its full size, 262,144 slots and a budget of 1e10 site updates, in both of its
    methods: coupled score-weighted pairs (B = 19073 progress units per slot, one-sweep window) and
    uncoupled systematic scan (B = 38146 draws per slot, b = 130, T = 1168).  Twelve slots spread
    over the run are recomputed one by one by the oracle (N*_p, retained cost, G vector)."""
    inst = synth.paper_shaped_config()
    P, budget = 262144, 1e10
    stride = P // 11 + 1
    k, ell = oracle.window_defaults(inst.n, 1)
    if method == "coupled-score":
        g = _gpu_run(ctx, inst, slots=P, budget_site_updates=budget, seed=4242, record_slots=True,
                     trace_stride=stride)
        B = synth.budget_horizon(budget, P)
        run = lambda p: oracle.coupled_run(k, ell, B, 4242, slot_offset=p)          # noqa: E731
        M = oracle.Model(inst)
    else:
        b = k - 1
        g = _gpu_run(ctx, inst, slots=P, budget_site_updates=budget, seed=4243, coupled=False,
                     scan=2, burn=b, length=ell - b, record_slots=True, trace_stride=stride)
        B = int(budget // P)
        run = lambda p: oracle.uncoupled_run(b, ell - b, B, 4243, slot_offset=p)    # noqa: E731
        M = oracle.Model(inst, scan=oracle.SCAN_SYSTEMATIC)
    assert g["stats"]["status"] == 0 and int(g["count"].sum()) == P
    for idx, p in enumerate(range(0, P, stride)):
        r = M.run_slots(run(p), 0, 1, 1, per_slot=True, slot_G=True)
        assert g["slot_nstar"][p] == r["slot_nstar"][0], p
        assert g["slot_S"][p] == r["slot_S"][0], p
        assert np.array_equal(g["trace_G"][idx], r["slot_G"][0]), p
