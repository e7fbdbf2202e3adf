"""The launch-shape cache of the batched decoder (host logic, no GPU): the first batch of a shape is
tuned and its choice stored; a later batch of the same shape bucket reuses it; retune tunes again."""
import json

from paper_2608_30239_gb300 import autotune


class FakeBatch:
    def __init__(self, n_inst, max_na, slots, classes=2, ext=0):
        self.info = [0] * 16
        self.info[1], self.info[2], self.info[3], self.info[9], self.info[11] = n_inst, slots, max_na, classes, ext
        self.tuned = 0
        self.shapes = []

    def autotune(self, est, se, candidates, reps):
        self.tuned += 1
        times = {c: 10.0 + i for i, c in enumerate(candidates)}
        return candidates[2], times

    def set_shape(self, warps, lanes):
        self.shapes.append((lanes, warps))


def test_tune_store_reuse_retune(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    a = FakeBatch(512, 4800, 524288)
    best, times, cached = autotune.tuned_shape(a, None, None, "GPU-X")
    assert (best, cached, a.tuned) == (autotune.DEFAULT_CANDIDATES[2], False, 1)
    with open(tmp_path / "cache.json") as f:
        stored = json.load(f)
    assert list(stored.values())[0]["shape"] == list(best)

    b = FakeBatch(500, 4100, 400000)                # same power-of-two buckets: reuses the choice
    assert autotune.shape_key("GPU-X", b) == autotune.shape_key("GPU-X", a)
    best_b, _, cached_b = autotune.tuned_shape(b, None, None, "GPU-X")
    assert cached_b and best_b == best and b.tuned == 0 and b.shapes == [best]

    c = FakeBatch(512, 4800, 524288, ext=1)         # caps or lags: a different kernel variant
    assert autotune.shape_key("GPU-X", c) != autotune.shape_key("GPU-X", a)
    assert autotune.shape_key("GPU-Y", a) != autotune.shape_key("GPU-X", a)

    _, _, cached_again = autotune.tuned_shape(a, None, None, "GPU-X", retune=True)
    assert not cached_again and a.tuned == 2
