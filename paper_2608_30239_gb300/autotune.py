"""Persisted launch-shape choices for batched decoding.

The tuner itself is native (mcpd_batch_autotune times candidate launch shapes on the batch);
this module remembers its choice (lanes per pair, warps per block) in a JSON cache keyed by GPU name and a coarse shape bucket
(instance count, largest n_active, total slots, size classes), so a batch of the same shape reuses
it.  Warps per block are an upper bound per size class: 0 lets every class take all that fit
(the 20-warp kernel variant where more than 12 fit), 12 keeps every class on the 12-warp variant.
"""
from __future__ import annotations

import json
import math
import os

from .build import BUILD

CACHE = os.path.join(BUILD, "autotune_cache.json")


def shape_key(gpu_name: str, batch) -> str:
    info = batch.info
    b = lambda v: 2 ** int(math.ceil(math.log2(max(1, int(v)))))   # noqa: E731
    return f"{gpu_name}|inst{b(info[1])}|na{b(info[3])}|slots{b(info[2])}|cls{int(info[9])}|ext{int(info[11])}"


def load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


DEFAULT_CANDIDATES = ((1, 0), (1, 12), (1, 6), (8, 0), (8, 12), (16, 0), (32, 0))


def tuned_shape(batch, est_dev, se_dev, gpu_name: str, candidates=DEFAULT_CANDIDATES, reps=1,
                retune=False):
    """Apply the cached (lanes per pair, warps per block) for this shape, or tune, store, apply."""
    cache = load()
    key = shape_key(gpu_name, batch)
    if not retune and key in cache:
        lanes, warps = cache[key]["shape"]
        batch.set_shape(int(warps), int(lanes))
        return (int(lanes), int(warps)), cache[key].get("times_ms", {}), True
    best, times = batch.autotune(est_dev, se_dev, candidates, reps)
    cache[key] = {"shape": list(best), "times_ms": {f"{a}x{b}": t for (a, b), t in times.items()}}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    return best, times, False
