"""The five-method comparison driver runs end to end on a small instance (needs a GB300)."""
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
                         "--slots", "2048", "--ref-burn", "50", "--ref-sweeps", "200", "--ref-chains", "2048"])
    rows = out["rows"]
    assert [r["method"] for r in rows] == ["SS", "RU", "SW", "cRU", "cSW"] * 2
    assert all(np.isfinite(r["mae_all"]) and np.isfinite(r["mae_top10"]) for r in rows)
    assert all(r["mean_tau_sweeps"] is not None and r["mean_tau_sweeps"] > 0 for r in rows if r["method"][0] == "c")
    assert all(r["site_updates"] > 0 for r in rows)
    assert len(out["reference"]["top10"]) == 10
