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
