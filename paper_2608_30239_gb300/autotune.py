"""Persisted launch-shape and slot-count choices for batched decoding.

Two levels:
  - launch shape (lanes per pair, warps per block): the tuner is native (mcpd_batch_autotune times
    candidate shapes on the batch); `tuned_shape` remembers its choice in a JSON cache keyed by GPU
    name and a coarse shape bucket (instance count, largest n_active, total slots, size classes),
    so a batch of the same shape reuses it.  Warps per block are an upper bound per size class: 0
    lets every class take all that fit (the 20-warp kernel variant where more than 12 fit), 12
    keeps every class on the 12-warp variant;
  - slots per instance at a fixed budget (`tuned_slots`): the estimator is unbiased for any number
    of slots P and horizon B (Theorem 2), so a workload that fixes each instance's budget P x B can
    take the P whose batch decodes fastest.  Each candidate is built, its shape tuned, one decode
    timed; the choice is cached by GPU name, instance-set bucket and candidate set.
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


def tuned_slots(ctx, instances, make_params, candidates, gpu_name: str, order_mode=1,
                shape_candidates=((1, 0), (1, 12)), retune=False):
    """Choose slots per instance: `make_params(P)` gives every instance's parameters with P slots
    (the caller keeps P x horizon fixed).  Returns (P, open batch built with it and shaped, its
    (lanes, warps), {P: decode ms}, cached).  Timing per candidate: one warm-up decode and one timed
    decode after its shape is applied."""
    from . import mcpd
    cache = load()
    b = lambda v: 2 ** int(math.ceil(math.log2(max(1, int(v)))))   # noqa: E731
    key = (f"{gpu_name}|slots-per-instance|inst{b(len(instances))}|"
           f"n{b(max(inst.n for inst in instances))}|cand{'-'.join(str(int(c)) for c in candidates)}")
    def build_and_shape(P):
        batch = mcpd.Batch(ctx, instances, make_params(P), order_mode=order_mode)
        est, se = _outputs(batch, ctx.device)
        shape, _, _ = tuned_shape(batch, est, se, gpu_name, shape_candidates)
        return batch, est, se, shape

    if not retune and key in cache:
        P = int(cache[key]["slots"])
        batch, _, _, shape = build_and_shape(P)
        return P, batch, shape, {int(k): v for k, v in cache[key]["times_ms"].items()}, True
    times, best = {}, None
    for P in candidates:
        batch, est, se, shape = build_and_shape(int(P))
        ms = []
        for _ in range(2):
            batch.run_async(est, se)
            ms.append(batch.collect(allow_step_limit=True)["kernel_ms"])
        times[int(P)] = ms[-1]
        if best is None or ms[-1] < times[best[0]]:
            if best is not None:
                best[1].close()
            best = (int(P), batch, shape)
        else:
            batch.close()
    cache = load()
    cache[key] = {"slots": best[0], "times_ms": {str(k): v for k, v in times.items()}}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    return best[0], best[1], best[2], times, False


def _outputs(batch, device):
    """Device arrays for a batch's estimates and standard errors."""
    import torch
    est = torch.empty(batch.total_active, dtype=torch.float64, device=f"cuda:{device}")
    return est, torch.empty_like(est)
