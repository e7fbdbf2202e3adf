"""Persisted launch-shape choices for batched decoding.

The tuner itself is native (mcpd_batch_autotune times candidate warps-per-block on the batch);
this module remembers its choice in a JSON cache keyed by GPU name and a coarse shape bucket
(instance count, largest n_active, total slots, coupled), so a batch of the same shape reuses it.
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
    return f"{gpu_name}|inst{b(info[1])}|na{b(info[3])}|slots{b(info[2])}"


def load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_shape(batch, est_dev, se_dev, gpu_name: str, candidates=(4, 6, 8, 12, 16), reps=1,
                retune=False):
    """Apply the cached warps-per-block for this shape, or tune, store and apply it."""
    cache = load()
    key = shape_key(gpu_name, batch)
    if not retune and key in cache:
        batch.set_shape(int(cache[key]["warps"]))
        return int(cache[key]["warps"]), cache[key].get("times_ms", {}), True
    best, times = batch.autotune(est_dev, se_dev, candidates, reps)
    cache[key] = {"warps": best, "times_ms": times}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    return best, times, False
