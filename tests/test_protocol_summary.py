"""The method-comparison program's per-cell summary over executions (host logic, no GPU)."""
import math

import numpy as np

from paper_2608_30239_gb300.protocol import _summary


def test_summary_mean_and_standard_error():
    rows = []
    vals = {("cSW", 1): [1.0, 2.0, 4.0], ("SS", 1): [3.0, 3.0, 3.0], ("cSW", 3): [5.0]}
    for (m, s), vs in vals.items():
        for e, v in enumerate(vs):
            rows.append({"execution": e, "sweeps": s, "method": m, "mae_all": v, "mae_top10": 2 * v,
                         "kernel_ms": 0.5})
    summ = {(c["sweeps"], c["method"]): c for c in _summary(rows)}
    c = summ[(1, "cSW")]
    assert c["n"] == 3 and math.isclose(c["mae_all"], 7 / 3)
    sd = math.sqrt(((1 - 7 / 3) ** 2 + (2 - 7 / 3) ** 2 + (4 - 7 / 3) ** 2) / 2)
    assert math.isclose(c["mae_all_se"], sd / math.sqrt(3))
    assert math.isclose(c["mae_top10"], 14 / 3) and math.isclose(c["mae_top10_se"], 2 * sd / math.sqrt(3))
    assert summ[(1, "SS")]["mae_all_se"] == 0.0
    assert summ[(3, "cSW")]["n"] == 1 and summ[(3, "cSW")]["mae_all_se"] is None
    assert np.isclose(summ[(3, "cSW")]["kernel_ms"], 0.5)


def test_protocol_windows_follow_table_s1():
    """The protocol's burn-in b = round_half_even(0.1 M) and averaging length M - b reproduce every
    printed value of Table S1 (tests/golden/table_s1.txt), e.g. b = 166 at M = 1665."""
    import os

    from paper_2608_30239_gb300.protocol import round_half_even
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_s1.txt")
    checked = 0
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            left, right = line.split("|")
            _, n_a, *bs = left.split()
            rest = [int(v) for v in right.split()]
            for s, b, mb in zip((1, 3, 5, 10, 20), (int(v) for v in bs), rest):
                M = s * int(n_a)
                assert round_half_even(0.1 * M) == b and M - round_half_even(0.1 * M) == mb, (n_a, s)
                checked += 1
    assert checked == 15


def test_scores_and_top_clones_on_hand_values():
    """All-clone MAE and top-10 MAE are plain means of absolute errors, over every clone and over the
    reference's largest marginals (ties to the lower position)."""
    from paper_2608_30239_gb300.protocol import scores, top_clones
    ref = np.array([0.0, 0.5, 0.4, 0.5, 0.1])
    est = np.array([0.1, 0.5, 0.2, 0.3, 0.1])
    top = top_clones(ref, 3)
    assert list(top) == [1, 3, 2]
    mae_all, mae_top = scores(est, ref, top)
    assert math.isclose(mae_all, (0.1 + 0.0 + 0.2 + 0.2 + 0.0) / 5)
    assert math.isclose(mae_top, (0.0 + 0.2 + 0.2) / 3)


def test_cell_parameters_follow_the_experimental_setup():
    """At n_a = 333 and s = 5: M = 1665 and b = 166 (Table S1); coupled k = b + 1 = 167, l = M, a
    20-sweep horizon and meeting cap; uncoupled b = 166, T = M - b = 1499 over twice the slots; the
    no-refill ablation has a horizon of zero; an uncapped run audits the cap without imposing it."""
    from paper_2608_30239_gb300 import mcpd
    from paper_2608_30239_gb300.protocol import cell_params
    c = cell_params("cSW", 5, 333, 1000)
    assert (c["k"], c["ell"], c["slots"], c["horizon"], c["meeting_cap"], c["tau_audit"]) == \
        (167, 1665, 1000, 20 * 333, 20 * 333, 20 * 333)
    assert c["coupled"] and c["scan"] == mcpd.MCPD_SCAN_SCORE and c["lag"] == 1 and c["n_active"] == 333
    u = cell_params("SS", 5, 333, 1000)
    assert (u["burn"], u["length"], u["slots"], u["horizon"]) == (166, 1499, 2000, 20 * 333)
    assert not u["coupled"] and u["scan"] == mcpd.MCPD_SCAN_SYSTEMATIC
    assert cell_params("cSW-nr", 1, 333, 1000)["horizon"] == 0
    assert cell_params("cRU", 1, 333, 1000)["scan"] == mcpd.MCPD_SCAN_UNIFORM
    assert "meeting_cap" not in cell_params("cSW", 1, 333, 1000, uncapped=True)
    assert cell_params("SW", 1, 333, 1000)["scan"] == mcpd.MCPD_SCAN_SCORE
