"""Batched decoding (many instances of uneven size in one launch) vs the CPU oracle, through the
C ABI (needs a GB300).  Each instance's integer bucket sums and finalized doubles must equal the
oracle's for that instance alone; graph replay, other launch shapes and another work order must
not change a bit."""
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
    stream = torch.cuda.Stream()
    c = mcpd.Context(0, stream=stream)
    c.torch_stream = stream
    yield c
    c.close()


def _uneven(count=7, seed=3):
    rng = synth.SplitMix64(seed)
    out = []
    for i in range(count):
        n = int(30 + rng.below(1, 570)[0])
        m = max(6, int(n / 13 + 0.5))
        k = int(3 + rng.below(1, 6)[0])
        npos = int(1 + rng.below(1, 4)[0])
        fp = 0.02 + 0.08 * float(rng.uniform(1)[0])
        fn = 0.05 + 0.15 * float(rng.uniform(1)[0])
        out.append(synth.make_instance(n, m, min(k, m), npos, fp, fn, npos / n, 900 + i, 950 + i))
    return out


def _params(insts, coupled=True):
    ps = []
    for i, inst in enumerate(insts):
        k, ell = oracle.window_defaults(inst.n, 1)
        if coupled:
            ps.append(dict(slots=300 + 97 * i, k=k, ell=ell, horizon=3 * ell + 11 * i, seed=77 + i,
                           instance_id=i))
        else:
            ps.append(dict(slots=200 + 31 * i, coupled=False, burn=k - 1, length=ell - k + 1,
                           horizon=4 * ell, seed=5 + i, instance_id=i))
    return ps


def _oracle(inst, kw):
    M = oracle.Model(inst)
    if kw.get("coupled", True):
        run = oracle.coupled_run(kw["k"], kw["ell"], kw["horizon"], kw["seed"], instance=kw["instance_id"],
                                 meeting_cap=kw.get("meeting_cap", 0), lag=kw.get("lag", 1))
        L = kw["ell"] - kw["k"] + 1
    else:
        run = oracle.uncoupled_run(kw["burn"], kw["length"], kw["horizon"], kw["seed"],
                                   instance=kw["instance_id"])
        L = kw["length"]
    res = M.run_slots(run, 0, kw["slots"], THREADS)
    res["est"], res["se"] = M.finalize(res, kw["slots"], L)
    return res


def _run(ctx, batch):
    import torch
    est = torch.empty(batch.total_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    with torch.cuda.stream(ctx.torch_stream):
        batch.run_async(est, se)
        st = batch.collect()
    return est.cpu().numpy(), se.cpu().numpy(), st


@pytest.mark.parametrize("coupled,classes", [(True, 1), (True, 3), (False, 1), (False, 3)])
def test_batch_matches_oracle_per_instance(ctx, coupled, classes):
    """Every instance equals the oracle alone, with one launch or with three size classes (each a
    launch fitted to its instances)."""
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven()
    ps = _params(insts, coupled)
    batch = mcpd.Batch(ctx, insts, ps, classes=classes)
    assert batch.classes == classes
    est, se, st = _run(ctx, batch)
    assert st["reps_retained"] > 0
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        ref = _oracle(inst, kw)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]), i
        assert np.array_equal(se[a:b], ref["se"]), i
    batch.close()


def test_graph_shapes_and_order_do_not_change_results(ctx):
    import torch
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(5, seed=9)
    ps = _params(insts)
    batch = mcpd.Batch(ctx, insts, ps)
    e0, s0, _ = _run(ctx, batch)
    est = torch.empty(batch.total_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    with torch.cuda.stream(ctx.torch_stream):
        batch.capture_graph(est, se)
        for _ in range(2):
            est.zero_()
            batch.launch_graph()
            batch.collect()
            assert np.array_equal(est.cpu().numpy(), e0)
            assert np.array_equal(se.cpu().numpy(), s0)
        best, times = batch.autotune(est, se, candidates=((1, 2), (1, 4), (8, 0), (16, 0), (32, 0)), reps=1)
    assert best in times and all(t > 0 for t in times.values())
    e1, s1, _ = _run(ctx, batch)
    assert np.array_equal(e1, e0) and np.array_equal(s1, s0)
    other = mcpd.Batch(ctx, insts, ps, order_mode=1)
    e2, s2, _ = _run(ctx, other)
    assert np.array_equal(e2, e0) and np.array_equal(s2, s0)
    split = mcpd.Batch(ctx, insts, ps, order_mode=1, classes=4)
    assert split.classes == 4
    e3, s3, _ = _run(ctx, split)
    assert np.array_equal(e3, e0) and np.array_equal(s3, s0)
    batch.close()
    other.close()
    split.close()


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_lane_groups_match_oracle(ctx, lanes):
    """G lanes per pair (ballot counting, XOR/ballot meeting, cooperative flushes): bit-identical
    to the oracle, including a random start and refill."""
    import torch
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(5, seed=13)
    ps = _params(insts)
    rng = np.random.default_rng(lanes)
    ps[1] = dict(ps[1], init_marginals=rng.random(insts[1].n) * 0.3)
    batch = mcpd.Batch(ctx, insts, ps, classes=2)
    batch.set_shape(0, lanes)
    assert int(batch.info[8]) == lanes and int(batch.info[9]) == 2
    est, se, st = _run(ctx, batch)
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        M = oracle.Model(inst, init_marginals=kw.get("init_marginals"))
        run = oracle.coupled_run(kw["k"], kw["ell"], kw["horizon"], kw["seed"], instance=kw["instance_id"])
        ref = M.run_slots(run, 0, kw["slots"], THREADS)
        ref["est"], ref["se"] = M.finalize(ref, kw["slots"], kw["ell"] - kw["k"] + 1)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (lanes, i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"])
    batch.close()


@pytest.mark.parametrize("lanes", [1, 16])
def test_batch_meeting_cap(ctx, lanes):
    """Meeting caps per instance (one instance uncapped) in one batch, one thread or a lane group
    per pair: every instance equals the oracle with its own cap."""
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(5, seed=21)
    ps = _params(insts)
    for i in range(len(ps)):
        if i != 2:
            ps[i] = dict(ps[i], meeting_cap=ps[i]["ell"] + 3 * i)
    batch = mcpd.Batch(ctx, insts, ps, classes=2)
    if lanes > 1:
        batch.set_shape(0, lanes)
    est, se, st = _run(ctx, batch)
    assert st["tau_over_audit"] > 0 and st["step_limit_hits"] == 0
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        ref = _oracle(inst, kw)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (lanes, i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"])
    batch.close()


@pytest.mark.parametrize("lanes", [1, 16])
def test_batch_lags(ctx, lanes):
    """Different lags per instance (1, 2, 5, 9, with a cap on one) in one batch, one thread or a
    lane group per pair: every instance equals the oracle; the site updates count each
    replication's pre-lag updates."""
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(4, seed=23)
    ps = _params(insts)
    lags = [1, 2, 5, 9]
    for i in range(len(ps)):
        ps[i] = dict(ps[i], lag=lags[i])
    ps[2] = dict(ps[2], meeting_cap=ps[2]["ell"] + 40)
    batch = mcpd.Batch(ctx, insts, ps, classes=2)
    if lanes > 1:
        batch.set_shape(0, lanes)
    est, se, st = _run(ctx, batch)
    started = 0
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        ref = _oracle(inst, kw)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (lanes, i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"])
    assert st["site_updates"] < 2 * st["progress_units"] - st["reps_started"]
    batch.close()


def test_batch_of_one_equals_single_instance_plan(ctx):
    import torch
    from paper_2608_30239_gb300 import mcpd
    inst = synth.high_noise_config()
    kw = dict(slots=2000, budget_site_updates=4e10 * 2000 / 524288, seed=20260)
    batch = mcpd.Batch(ctx, [inst], [kw])
    e, s, st = _run(ctx, batch)
    plan = mcpd.Plan(ctx, inst, **kw)
    pe = torch.empty(plan.n_active, dtype=torch.float64, device="cuda:0")
    ps = torch.empty_like(pe)
    with torch.cuda.stream(ctx.torch_stream):
        plan.run_async(pe, ps)
        pst = plan.collect()
    assert np.array_equal(pe.cpu().numpy(), e) and np.array_equal(ps.cpu().numpy(), s)
    assert pst["site_updates"] == st["site_updates"]
    batch.close()
    plan.close()


def test_paper_sized_batch_runs(ctx):
    """32 instances drawn like the 512-instance workload (n in [200, 5000]), 256 slots each, 20
    sweeps of horizon: completes, every instance finite, sampled instances match the oracle."""
    from paper_2608_30239_gb300 import mcpd
    insts = synth.batched_configs(32, seed=11)
    ps = [dict(slots=256, horizon=20 * inst.n, seed=1000 + i, instance_id=i) for i, inst in enumerate(insts)]
    batch = mcpd.Batch(ctx, insts, ps, order_mode=1)
    est, se, st = _run(ctx, batch)
    assert np.all(np.isfinite(est)) and np.all(se >= 0)
    for i in (0, 7):
        inst = insts[i]
        k, ell = oracle.window_defaults(inst.n, 1)
        ref = _oracle(inst, dict(ps[i], k=k, ell=ell))
        got = batch.buckets(i)
        assert np.array_equal(got["S1"], ref["S1"]) and np.array_equal(got["count"], ref["count"])
    batch.close()


@pytest.mark.parametrize("lanes", [1, 8, 32])
def test_batch_mixed_degree_instances(ctx, lanes):
    """Instances whose clones sit in different numbers of pools (padded rows), next to uniform
    ones, with a random start on one: every launch shape equals the oracle per instance."""
    from paper_2608_30239_gb300 import mcpd
    insts = [synth.make_mixed_instance(180 + 40 * i, 17 + 2 * i, 2, 7, 4, 0.08, 0.18, 4 / (180 + 40 * i),
                                       600 + i, 700 + i) for i in range(3)] + _uneven(2, seed=21)
    ps = _params(insts)
    ps[0] = dict(ps[0], init_marginals=np.random.default_rng(9).random(insts[0].n) * 0.25)
    batch = mcpd.Batch(ctx, insts, ps, classes=2)
    if lanes != 1:
        batch.set_shape(0, lanes)
    est, se, st = _run(ctx, batch)
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        M = oracle.Model(inst, init_marginals=kw.get("init_marginals"))
        run = oracle.coupled_run(kw["k"], kw["ell"], kw["horizon"], kw["seed"], instance=kw["instance_id"])
        ref = M.run_slots(run, 0, kw["slots"], THREADS)
        ref["est"], ref["se"] = M.finalize(ref, kw["slots"], kw["ell"] - kw["k"] + 1)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (lanes, i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"])
    batch.close()


@pytest.mark.parametrize("classes", [1, 2])
def test_batch_few_slots_per_instance(ctx, classes):
    """One to three slots per instance, so that a warp's few live lanes hold slots of different
    instances (2 to 16 bit words per column, mixed degrees) and leave while others go on: the work
    the live lanes share at a replication's start and end reads the ending lane's own instance.
    Refill with a horizon of three windows, a random start on two instances; every instance
    equals the oracle."""
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(5, seed=31) + [synth.make_mixed_instance(40 + 150 * i, 9 + 3 * i, 2, 7, 3, 0.08, 0.18,
                                                             3 / (40 + 150 * i), 820 + i, 830 + i)
                                   for i in range(3)]
    ps = []
    for i, inst in enumerate(insts):
        k, ell = oracle.window_defaults(inst.n, 1)
        ps.append(dict(slots=1 + i % 3, k=k, ell=ell, horizon=3 * ell + 7 * i, seed=901 + i, instance_id=i))
    ps[1] = dict(ps[1], init_marginals=np.random.default_rng(31).random(insts[1].n) * 0.3)
    ps[6] = dict(ps[6], init_marginals=np.random.default_rng(32).random(insts[6].n) * 0.3)
    batch = mcpd.Batch(ctx, insts, ps, classes=classes)
    est, se, st = _run(ctx, batch)
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        M = oracle.Model(inst, init_marginals=kw.get("init_marginals"))
        run = oracle.coupled_run(kw["k"], kw["ell"], kw["horizon"], kw["seed"], instance=kw["instance_id"])
        ref = M.run_slots(run, 0, kw["slots"], THREADS)
        ref["est"], ref["se"] = M.finalize(ref, kw["slots"], kw["ell"] - kw["k"] + 1)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (classes, i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"], equal_nan=True)
    batch.close()


def test_batch_systematic_uncoupled(ctx):
    """Uncoupled systematic-scan chains (Algorithm 1) in a batch of uneven instances, two classes."""
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(4, seed=31)
    ps = [dict(slots=150 + 40 * i, coupled=False, scan=mcpd.MCPD_SCAN_SYSTEMATIC, burn=inst.n // 10,
               length=inst.n, horizon=3 * inst.n, seed=61 + i, instance_id=i) for i, inst in enumerate(insts)]
    batch = mcpd.Batch(ctx, insts, ps, classes=2)
    est, se, st = _run(ctx, batch)
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        M = oracle.Model(inst, scan=oracle.SCAN_SYSTEMATIC)
        run = oracle.uncoupled_run(kw["burn"], kw["length"], kw["horizon"], kw["seed"], instance=i)
        ref = M.run_slots(run, 0, kw["slots"], THREADS)
        ref["est"], ref["se"] = M.finalize(ref, kw["slots"], kw["length"])
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"])
    batch.close()


@pytest.mark.parametrize("capped", [False, True])
@pytest.mark.parametrize("deg", [3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("warps", [0, 12, 20])
def test_uniform_degree_batches(ctx, deg, warps, capped):
    """Coupled batches whose instances all sit in `deg` pools per clone launch the build with that
    compile-time degree (mask-indexed thresholds up to degree 6; info[12]), and with meeting caps
    the capped build of that degree; every instance, of its own size, rates, window, random start
    or scan weights, equals the oracle alone, in the 12-warp build and the 20-warp one."""
    from paper_2608_30239_gb300 import mcpd
    insts, ps = [], []
    rng = np.random.default_rng(deg)
    for i in range(5):
        n = 120 + 173 * i
        inst = synth.make_instance(n, max(deg + 2, n // 13), deg, 1 + i % 3, 0.03 + 0.02 * i, 0.1 + 0.03 * i,
                                   (1 + i % 3) / n, 60 + i, 70 + i)
        k, ell = oracle.window_defaults(n, 1)
        kw = dict(slots=400 + 61 * i, k=k, ell=ell, horizon=3 * ell + 7 * i, seed=90 + i, instance_id=i)
        if capped and i != 2:
            kw["meeting_cap"] = ell + 5 * i
        if i == 1:
            kw["init_marginals"] = rng.uniform(0.0, 0.2, n)
        if i == 3:
            kw.update(scan=mcpd.MCPD_SCAN_CUSTOM, scan_weights=rng.uniform(0.5, 2.0, n))
        insts.append(inst)
        ps.append(kw)
    batch = mcpd.Batch(ctx, insts, ps, classes=1)
    if warps:
        batch.set_shape(warps)
    assert int(batch.info[12]) == 1
    est, se, st = _run(ctx, batch)
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        M = oracle.Model(inst, scan=kw.get("scan", oracle.SCAN_SCORE), custom_w=kw.get("scan_weights"),
                         init_marginals=kw.get("init_marginals"))
        run = oracle.coupled_run(kw["k"], kw["ell"], kw["horizon"], kw["seed"], instance=kw["instance_id"],
                                 meeting_cap=kw.get("meeting_cap", 0))
        ref = M.run_slots(run, 0, kw["slots"], THREADS)
        ref["est"], ref["se"] = M.finalize(ref, kw["slots"], kw["ell"] - kw["k"] + 1)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"]), i
    batch.close()


def test_automatic_classes_follow_uniform_degree(ctx):
    """With the number of classes left to the library, coupled instances of one uniform degree
    get classes of their own (each launching the build of its degree, info[12]); mixed-degree
    instances stay in the generic build. Every instance equals the oracle."""
    from paper_2608_30239_gb300 import mcpd
    insts = [synth.make_instance(150 + 90 * i, 14 + i, d, 2, 0.05, 0.12, 2 / (150 + 90 * i), 970 + i, 980 + i)
             for i, d in enumerate([4, 7, 4, 5, 7, 4])]
    insts.append(synth.make_mixed_instance(260, 21, 2, 7, 3, 0.08, 0.18, 3 / 260, 990, 991))
    ps = _params(insts)
    for i in (0, 4):
        ps[i] = dict(ps[i], meeting_cap=ps[i]["ell"] + 11)
    batch = mcpd.Batch(ctx, insts, ps)
    # degree groups 4, 5, 7 and the mixed instance: at least one class each, three with a degree build
    assert batch.classes >= 4 and int(batch.info[12]) >= 3
    est, se, st = _run(ctx, batch)
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        ref = _oracle(inst, kw)
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(est[a:b], ref["est"]) and np.array_equal(se[a:b], ref["se"])
    batch.close()


def test_batch_extension_by_slot_ranges(ctx):
    """mcpd_batch_extend_async: every instance (or the masked ones) runs its next P_i slots into the
    same buckets; each instance then equals the oracle over all its slots, an instance left out
    keeps its estimate, and a later run or graph launch starts again from the first slot."""
    from paper_2608_30239_gb300 import mcpd
    insts = _uneven(6, seed=9)
    ps = _params(insts)
    batch = mcpd.Batch(ctx, insts, ps, classes=2)
    e0, s0, _ = _run(ctx, batch)
    import torch
    est = torch.empty(batch.total_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    mask = np.array([1, 0, 1, 1, 0, 1], np.int32)
    ranges = np.ones(len(insts), np.int64)
    with torch.cuda.stream(ctx.torch_stream):
        for m in (None, mask):
            batch.extend_async(est, se, m)
            batch.collect()
            ranges += 1 if m is None else m
    got_e, got_s = est.cpu().numpy(), se.cpu().numpy()
    for i, (inst, kw) in enumerate(zip(insts, ps)):
        total = kw["slots"] * int(ranges[i])
        ref = _oracle(inst, dict(kw, slots=total))
        got = batch.buckets(i)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(got_e[a:b], ref["est"]) and np.array_equal(got_s[a:b], ref["se"]), i
    e1, s1, _ = _run(ctx, batch)                     # a plain run starts from the first slot again
    assert np.array_equal(e1, e0) and np.array_equal(s1, s0)
    with torch.cuda.stream(ctx.torch_stream):
        batch.extend_async(est, se)
        batch.collect()
        batch.capture_graph(est, se)                  # capture and launch restore the first range
        batch.launch_graph()
        batch.collect()
    assert np.array_equal(est.cpu().numpy(), e0)
    batch.close()


def test_batched_workload_full_size(ctx):
    """The batched workload at its full size, as the bench decodes it: 512 uneven instances (n in
    [200, 5000], k in 4..8, rates and positives per instance), 2048 slots each with a 10-sweep
    horizon and the paper's 20-sweep meeting cap, automatic classes (by degree, then size) running
    concurrently, in a captured graph.  The four smallest instances equal the oracle alone bit for bit (buckets and
    doubles); every instance's estimates are finite, in the valid range of an unbiased estimator's
    mean of bounded corrections, and every slot is counted once."""
    import torch
    from paper_2608_30239_gb300 import mcpd
    insts = synth.batched_configs(512, seed=11)
    ps = [dict(slots=2048, horizon=10 * inst.n, seed=5000 + i, instance_id=i, meeting_cap=20 * inst.n)
          for i, inst in enumerate(insts)]
    batch = mcpd.Batch(ctx, insts, ps, order_mode=1)
    # every instance sits in the same number of pools per clone: every class launches the build
    # of its degree
    assert batch.classes >= 4 and int(batch.info[12]) == batch.classes
    est = torch.empty(batch.total_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    with torch.cuda.stream(ctx.torch_stream):
        batch.capture_graph(est, se)
        batch.launch_graph()
        st = batch.collect()
    e, s = est.cpu().numpy(), se.cpu().numpy()
    assert st["status"] == 0 and np.all(np.isfinite(e)) and np.all(s >= 0)
    for i in range(len(insts)):
        assert int(batch.buckets(i)["count"].sum()) == 2048
    for i in np.argsort([inst.n for inst in insts], kind="stable")[:4]:
        inst, kw = insts[i], ps[i]
        k, ell = oracle.window_defaults(inst.n, 1)
        M = oracle.Model(inst)
        run = oracle.coupled_run(k, ell, kw["horizon"], kw["seed"], instance=kw["instance_id"],
                                 meeting_cap=kw["meeting_cap"])
        ref = M.run_slots(run, 0, kw["slots"], THREADS)
        ref["est"], ref["se"] = M.finalize(ref, kw["slots"], ell - k + 1)
        got = batch.buckets(int(i))
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            assert np.array_equal(got[key], ref[key]), (i, key)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert np.array_equal(e[a:b], ref["est"]) and np.array_equal(s[a:b], ref["se"]), i
    batch.close()
