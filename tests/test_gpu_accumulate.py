"""mcpd_run_slots_async: a fixed-budget estimate extended slot range by slot range (needs a GB300).

Theorem 2 treats the P slot means as i.i.d.; the library keys every random number by the global
slot id and sums slots into integer N*_p buckets, so runs over consecutive slot ranges added into
the same buckets must give, bit for bit, the buckets and the finalized doubles of one run over all
those slots with the same horizon, and both must equal the CPU oracle's."""
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


def _out(plan):
    import torch
    est = torch.full((plan.n_active,), float("nan"), dtype=torch.float64, device="cuda:0")
    return est, torch.full_like(est, float("nan"))


def _collect(plan, est, se):
    st = plan.collect()
    out = dict(est=est.cpu().numpy(), se=se.cpu().numpy(), stats=st)
    out.update(plan.buckets())
    return out


def _same(a, b):
    for key in ("S1", "S2_lo", "S2_hi", "count"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(a["est"], b["est"])
    assert np.array_equal(a["se"], b["se"], equal_nan=True)


@pytest.mark.parametrize("chunks", [(1000, 2333, 1), (4096, 4096, 4096), (7, 1, 5000)])
def test_ranges_equal_one_run_and_the_oracle(ctx, chunks):
    """Ragged ranges (one slot, a few slots, several rounds of the GPU's pairs) on a refilling
    medium design: every partial total equals one run over as many slots and the oracle."""
    from paper_2608_30239_gb300 import mcpd
    inst = synth.make_instance(300, 24, 5, 3, 0.05, 0.15, 3 / 300, 501, 502)
    k, ell, B, seed = 31, 300, 1200, 4242
    plan = mcpd.Plan(ctx, inst, slots=max(chunks), k=k, ell=ell, horizon=B, seed=seed)
    est, se = _out(plan)
    M = oracle.Model(inst)
    total = 0
    for i, n in enumerate(chunks):
        plan.run_slots_async(n, est, se, accumulate=i > 0)
        got = _collect(plan, est, se)
        total += n
        assert got["stats"]["status"] == 0
        assert int(got["count"].sum()) == total
        one = mcpd.Plan(ctx, inst, slots=total, k=k, ell=ell, horizon=B, seed=seed)
        e1, s1 = _out(one)
        one.run_async(e1, s1)
        ref = _collect(one, e1, s1)
        one.close()
        _same(got, ref)
        o = M.run_slots(oracle.coupled_run(k, ell, B, seed), 0, total, THREADS)
        o["est"], o["se"] = M.finalize(o, total, ell - k + 1)
        _same(got, o)
    plan.close()


def test_ranges_with_lag_cap_and_random_start(ctx):
    """The kernel variant with a meeting cap and a lag, from a random start, over two ranges."""
    from paper_2608_30239_gb300 import mcpd
    inst = synth.make_instance(120, 12, 4, 2, 0.05, 0.1, 2 / 120, 61, 62)
    nu = np.random.default_rng(3).uniform(0.0, 0.3, inst.n)
    k, ell, B, seed, cap, lag = 13, 120, 500, 99, 240, 3
    plan = mcpd.Plan(ctx, inst, slots=3000, k=k, ell=ell, horizon=B, seed=seed, init_marginals=nu,
                     meeting_cap=cap, lag=lag)
    est, se = _out(plan)
    plan.run_slots_async(1234, est, se)
    plan.collect()
    plan.run_slots_async(3000, est, se, accumulate=True)
    got = _collect(plan, est, se)
    plan.close()
    M = oracle.Model(inst, init_marginals=nu)
    o = M.run_slots(oracle.coupled_run(k, ell, B, seed, meeting_cap=cap, lag=lag), 0, 4234, THREADS)
    o["est"], o["se"] = M.finalize(o, 4234, ell - k + 1)
    _same(got, o)


def test_full_size_ranges_equal_one_launch(ctx):
    """The bench's workload (1298 x 97, high noise) in the launch shape the bench times: two ranges
    of 262144 slots equal one run of 524288 slots with the same horizon."""
    from paper_2608_30239_gb300 import mcpd
    inst = synth.high_noise_config()
    B = synth.budget_horizon(4e10, 524288)
    one = mcpd.Plan(ctx, inst, slots=524288, horizon=B, seed=20260)
    e1, s1 = _out(one)
    one.run_async(e1, s1)
    ref = _collect(one, e1, s1)
    plan = mcpd.Plan(ctx, inst, slots=524288, horizon=B, seed=20260)
    est, se = _out(plan)
    plan.run_slots_async(262144, est, se)
    plan.collect()
    plan.run_slots_async(262144, est, se, accumulate=True)
    got = _collect(plan, est, se)
    assert got["stats"]["resident_pairs"] <= one.info[8]
    _same(got, ref)
    one.close()
    plan.close()


def test_invalid_ranges_are_refused(ctx):
    from paper_2608_30239_gb300 import mcpd
    inst = synth.tiny_config(1)
    plan = mcpd.Plan(ctx, inst, slots=64, k=3, ell=20, horizon=60, seed=1)
    est, se = _out(plan)
    with pytest.raises(mcpd.McpdError) as ei:           # nothing to add onto yet
        plan.run_slots_async(10, est, se, accumulate=True)
    assert ei.value.code == mcpd.MCPD_EINVAL
    with pytest.raises(mcpd.McpdError) as ei:
        plan.run_slots_async(0, est, se)
    assert ei.value.code == mcpd.MCPD_EINVAL
    plan.close()
    rec = mcpd.Plan(ctx, inst, slots=64, k=3, ell=20, horizon=60, seed=1, record_slots=True)
    rec.run_slots_async(64, est, se)
    rec.collect()
    with pytest.raises(mcpd.McpdError) as ei:           # per-slot records cover one run
        rec.run_slots_async(10, est, se, accumulate=True)
    assert ei.value.code == mcpd.MCPD_EINVAL
    rec.close()
