"""Host-side training targets of the learned scan weights (numpy, no GPU)."""
import numpy as np

from paper_2608_30239_gb300.learned import segments, weight_target


class _I:
    def __init__(self, n):
        self.n = n


def test_weight_targets_are_per_instance_distributions():
    seg = segments([_I(3), _I(4)])
    assert seg.tolist() == [0, 3, 7]
    p = np.array([0.0, 0.5, 1.0, -0.2, 0.1, 0.9, 1.3])        # unbiased estimates may leave [0, 1]
    for mode in ("uncertainty", "positive"):
        w = weight_target(p, seg, floor=0.01, mode=mode)
        assert (w > 0).all()
        assert np.isclose(w[0:3].sum(), 1.0) and np.isclose(w[3:7].sum(), 1.0)
    u = weight_target(p, seg, floor=0.01, mode="uncertainty")
    assert u[1] > u[0] and np.isclose(u[0], u[2])               # p(1 - p) peaks at 1/2
    assert np.isclose(u[3], u[6])                               # clipped to 0 and to 1 alike
    pos = weight_target(p, seg, floor=0.01, mode="positive")
    assert pos[2] > pos[1] > pos[0] and pos[6] > pos[5] > pos[4] > pos[3]


def test_time_to_se_extends_until_the_target(monkeypatch):
    """The measured time to a target SE (learned.time_to_se), driven by a stand-in plan whose largest
    SE falls as 0.5 / sqrt(P): the first range has first_slots slots, later ones are sized by the
    P^-1/2 law (at most 8x the slots so far, whole warps of 32), every range after the first adds
    to the same estimate, the kernel time is the sum over ranges, and the run stops at the first
    range that meets the target."""
    import math

    from paper_2608_30239_gb300 import learned, mcpd
    calls = []

    class Plan:
        def __init__(self, ctx, inst, **kw):
            self.n_active, self.total = inst.n, 0
            self.kw = kw

        def run_slots_async(self, slots, est, se, accumulate=False):
            assert accumulate == (self.total > 0)
            self.total = self.total + slots if accumulate else slots
            calls.append(slots)
            se.fill_(0.5 / math.sqrt(self.total))

        def collect(self):
            return {"kernel_ms": 1.0 * calls[-1], "sum_tau": 0, "reps_retained": 1}

        def close(self):
            pass

    import torch
    monkeypatch.setattr(mcpd, "Plan", Plan)
    monkeypatch.setattr(torch, "empty", lambda n, dtype=None, device=None: torch.zeros(n, dtype=dtype))
    r = learned.time_to_se(type("Ctx", (), {"device": 0})(), _I(50), target=0.005, first_slots=1024)
    need = (0.5 / 0.005) ** 2                                   # 10,000 slots
    assert r["met"] and r["slots"] >= need and r["path"][-1][1] <= 0.005
    assert all(p[1] > 0.005 for p in r["path"][:-1])            # stopped at the first that met it
    assert calls[0] == 1024 and all(c % 32 == 0 for c in calls[1:])
    assert all(calls[i + 1] <= 8 * sum(calls[:i + 1]) for i in range(len(calls) - 1))
    assert r["kernel_ms"] == sum(calls) and r["ranges"] == len(calls)
    assert r["slots"] < 2 * need                                # the law sizes the last range
