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
        return candidates[min(2, len(candidates) - 1)], times

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


def test_slots_per_instance_tuner(tmp_path, monkeypatch):
    """The slot-count tuner builds one batch per candidate P (parameters from the caller, who keeps
    P x horizon fixed), keeps the fastest, closes the others, caches the choice and, on a later call,
    builds only the cached P."""
    from paper_2608_30239_gb300 import mcpd
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    built, closed = [], []
    ms_of = {512: 9.0, 1024: 7.0, 2048: 8.0}

    class Batch(FakeBatch):
        def __init__(self, ctx, insts, params, order_mode=0):
            super().__init__(len(insts), 4800, len(insts) * params[0]["slots"])
            self.P = params[0]["slots"]
            built.append(self.P)

        def run_async(self, est, se):
            pass

        def collect(self, allow_step_limit=False):
            return {"kernel_ms": ms_of[self.P]}

        def close(self):
            closed.append(self.P)

    class Inst:
        n = 1000

    monkeypatch.setattr(mcpd, "Batch", Batch)
    monkeypatch.setattr(autotune, "_outputs", lambda batch, device: (None, None))
    ctx = type("Ctx", (), {"device": 0})()
    make = lambda P: [dict(slots=P, horizon=20 * 1024 // P)] * 3   # noqa: E731
    P, batch, shape, times, cached = autotune.tuned_slots(ctx, [Inst()] * 3, make, (512, 1024, 2048), "GPU-X")
    assert (P, cached, batch.P) == (1024, False, 1024)
    assert built == [512, 1024, 2048] and sorted(closed) == [512, 2048]
    assert times == ms_of
    built.clear()
    P2, batch2, _, times2, cached2 = autotune.tuned_slots(ctx, [Inst()] * 3, make, (512, 1024, 2048), "GPU-X")
    assert (P2, cached2, built) == (1024, True, [1024]) and times2 == ms_of
