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
