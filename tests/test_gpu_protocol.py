"""The method comparison program (five methods and the no-refill ablation) runs end to end on a small instance (needs a GB300)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_protocol_small():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_30239_gb300 import build, protocol
    build.build()
    out = protocol.main(["--n", "200", "--m", "20", "--deg", "3", "--n-active", "100", "--sweeps", "1,3",
                         "--slots", "2048", "--ref-burn", "50", "--ref-sweeps", "200", "--ref-chains", "2048",
                         "--executions", "2"])
    rows = out["rows"]
    assert [r["method"] for r in rows] == ["SS", "RU", "SW", "cRU", "cSW", "cSW-nr"] * 4
    assert [r["execution"] for r in rows] == [0] * 12 + [1] * 12
    summ = out["summary"]
    assert len(summ) == 12 and all(c["n"] == 2 and c["mae_all_se"] is not None for c in summ)
    first = {(r["sweeps"], r["method"]): r["mae_all"] for r in rows if r["execution"] == 0}
    second = {(r["sweeps"], r["method"]): r["mae_all"] for r in rows if r["execution"] == 1}
    assert first != second                 # new seeds per execution
    assert all(np.isfinite(r["mae_all"]) and np.isfinite(r["mae_top10"]) for r in rows)
    assert all(r["mean_tau_sweeps"] is not None and r["mean_tau_sweeps"] > 0 for r in rows if r["method"][0] == "c")
    assert all(r["site_updates"] > 0 for r in rows)
    assert len(out["reference"]["top10"]) == 10
    assert out["meeting_cap_sweeps"] == 20
    for r in rows:
        if r["method"][0] == "c":      # the cap is imposed: the audited hits are pairs attempted
            assert 0 <= r["cap_hits"] <= r["reps_started"] and r["step_limit_hits"] == 0
    for r in rows:                     # without refill every slot keeps exactly one pair
        if r["method"] == "cSW-nr":
            assert r["reps_retained"] == 2048
        elif r["method"] == "cSW":
            assert r["reps_retained"] > 2048


@pytest.mark.parametrize("method", ["cSW", "SS", "cRU", "SW", "cSW-nr"])
def test_protocol_cell_equals_the_oracle(method):
    """One cell of the comparison (estimator length 1 sweep, the paper's instance shape: 3 pools
    per clone, q = 2.6 / n, pruned) decoded by the program's own path gives, bit for bit, the
    estimate vector of the CPU oracle run with the same cell parameters, and so the same scores."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os

    import oracle
    import synth
    from paper_2608_30239_gb300 import build, mcpd, protocol
    build.build()
    inst = synth.make_instance(260, 20, 3, 3, 0.10, 0.10, 2.6 / 260, 5007, 9007)
    kw = protocol.cell_params(method, 1, 90, 512)
    ctx = mcpd.Context(0)
    est, active, st = protocol._decode(ctx, inst, seed=77, **kw)
    ctx.close()
    scan = {mcpd.MCPD_SCAN_SCORE: oracle.SCAN_SCORE, mcpd.MCPD_SCAN_UNIFORM: oracle.SCAN_UNIFORM,
            mcpd.MCPD_SCAN_SYSTEMATIC: oracle.SCAN_SYSTEMATIC}[kw["scan"]]
    if kw["coupled"]:
        ref = oracle.decode(inst, kw["slots"], kw["k"], kw["ell"], kw["horizon"], seed=77, threads=os.cpu_count(),
                            n_active=90, scan=scan, meeting_cap=kw.get("meeting_cap", 0))
    else:
        ref = oracle.decode(inst, kw["slots"], 0, 0, kw["horizon"], seed=77, threads=os.cpu_count(), n_active=90,
                            scan=scan, coupled=False, burn=kw["burn"], length=kw["length"])
    assert np.array_equal(est, ref["est"])
    other = np.linspace(0.0, 0.5, len(est))
    top = protocol.top_clones(other)
    assert protocol.scores(est, other, top) == protocol.scores(ref["est"], other, top)
