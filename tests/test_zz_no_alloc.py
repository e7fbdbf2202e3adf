"""mcpd_decode_noalloc, the entry point for callers that may not allocate device memory.

Some callers cannot call cudaMalloc or cudaFree: a component inside an application or server that
owns all device memory through its own pool allocator and gives each part a fixed budget, or a host
loop that cannot afford the synchronisation those calls can imply.  For them the library offers a
decode whose scratch lives in a 64 MiB array compiled into the library.  This file checks, through
the C ABI, that it returns exactly what the allocating path returns, on two calls in a row (the
array is reused and must be cleared by each call), and that a problem too large for the array is
refused cleanly.  It is named so that pytest collects it after every other test file.
"""
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


def _plan_path(ctx, inst, **kw):
    import torch
    from paper_2608_30239_gb300 import mcpd
    plan = mcpd.Plan(ctx, inst, **kw)
    est = torch.empty(plan.n_active, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    plan.run_async(est, se)
    st = plan.collect()
    out = (est.cpu().numpy(), se.cpu().numpy(), st)
    plan.close()
    return out


def _noalloc_path(ctx, inst, **kw):
    import torch
    from paper_2608_30239_gb300 import mcpd
    na = int(mcpd.mcpd_inspect(inst, **kw)["info"][0])
    est = torch.full((na,), float("nan"), dtype=torch.float64, device="cuda:0")
    se = torch.full_like(est, float("nan"))
    st = ctx.decode_noalloc(inst, est, se, **kw)
    return est.cpu().numpy(), se.cpu().numpy(), st


CASES = {
    "medium-refill": (lambda: synth.make_instance(400, 31, 5, 3, 0.05, 0.1, 3 / 400, 41, 42),
                      dict(slots=7777, k=41, ell=400, horizon=2017, seed=2024)),
    "library-high-noise": (lambda: synth.high_noise_config(),
                           dict(slots=4096, budget_site_updates=4e10 * 4096 / 524288, seed=20260)),
    "capped-lag": (lambda: synth.make_instance(400, 31, 5, 3, 0.05, 0.1, 3 / 400, 43, 44),
                   dict(slots=5000, k=41, ell=400, horizon=1600, seed=77, meeting_cap=800, lag=2)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_equals_allocating_path_twice(ctx, case):
    make, kw = CASES[case]
    inst = make()
    e_ref, s_ref, st_ref = _plan_path(ctx, inst, **kw)
    for call in range(2):
        e, s, st = _noalloc_path(ctx, inst, **kw)
        assert st["status"] == 0
        assert np.array_equal(e, e_ref), (case, call)
        assert np.array_equal(s, s_ref), (case, call)
        assert st["reps_retained"] == st_ref["reps_retained"]
        assert st["site_updates"] == st_ref["site_updates"]
        assert 0 < st["resident_pairs"] <= st_ref["resident_pairs"]
    if case == "library-high-noise":
        # 1298 clones need about 21 KB of pair accumulators per pair: the 64 MiB array holds fewer
        # pairs than the allocating path runs, and the results above were still identical
        assert st["resident_pairs"] < st_ref["resident_pairs"]


def test_noalloc_refuses_outputs_not_on_the_device(ctx):
    """Host arrays passed as outputs are refused before any launch; the context stays usable."""
    import torch
    from paper_2608_30239_gb300 import mcpd
    inst = synth.tiny_config(1)
    kw = dict(slots=256, k=3, ell=20, horizon=60, seed=5)
    est = torch.zeros(inst.n, dtype=torch.float64)
    se = torch.zeros_like(est)
    with pytest.raises(mcpd.McpdError) as ei:
        ctx.decode_noalloc(inst, est, se, **kw)
    assert ei.value.code == mcpd.MCPD_EINVAL
    e, s, st = _noalloc_path(ctx, inst, **kw)
    e_ref, s_ref, _ = _plan_path(ctx, inst, **kw)
    assert np.array_equal(e, e_ref) and np.array_equal(s, s_ref)


def test_noalloc_rejects_problems_beyond_its_array(ctx):
    from paper_2608_30239_gb300 import mcpd
    inst = synth.high_noise_config()
    import torch
    est = torch.empty(inst.n, dtype=torch.float64, device="cuda:0")
    se = torch.empty_like(est)
    # 4000 N*_p buckets of 1298 clones need 4000 * 1298 * 24 bytes > 64 MiB
    with pytest.raises(mcpd.McpdError) as ei:
        ctx.decode_noalloc(inst, est, se, slots=64, k=0, ell=1298, horizon=4000 * 1298)
    assert ei.value.code == mcpd.MCPD_ETOO_LARGE
    # the context and the array are still usable afterwards
    e, s, st = _noalloc_path(ctx, synth.tiny_config(1), slots=512, k=3, ell=20, horizon=60, seed=3)
    M = oracle.Model(synth.tiny_config(1))
    ref = M.run_slots(oracle.coupled_run(3, 20, 60, seed=3), 0, 512, 4)
    e_ref, s_ref = M.finalize(ref, 512, 18)
    assert np.array_equal(e, e_ref) and np.array_equal(s, s_ref)
