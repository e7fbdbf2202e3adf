"""The same draws through the single-instance kernel and through the batch kernel.

  python -m paper_2608_30239_gb300.kernel_compare {plan|batch1|batch128|all}

The high-noise bench instance (1298 clones x 97 pools, 6 pools per clone), 87,552 slots, B = 38146:
`plan` decodes it with a Plan (tables staged in shared memory, compile-time degree), `batch1` as a
Batch of that one instance, `batch128` as a Batch of 128 copies (684 slots each, seeds per copy),
one size class.  Each configuration is launched three times; prints one JSON line with the
fastest kernel time, the draws (progress units) and the batch's launch facts.
"""
from __future__ import annotations

import argparse
import json

import synth

from . import build, mcpd

P, B = 87552, 38146


def _plan(ctx, stream, inst):
    import torch
    plan = mcpd.Plan(ctx, inst, slots=P, horizon=B, seed=20260)
    est = torch.empty(plan.n_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    ms = []
    with torch.cuda.stream(stream):
        for _ in range(3):
            plan.run_async(est, se)
            st = plan.collect()
            ms.append(st["kernel_ms"])
    plan.close()
    return dict(ms=min(ms), draws=st["progress_units"])


def _batch(ctx, stream, inst, copies):
    import torch
    params = [dict(slots=P // copies, horizon=B, seed=20260 + i, instance_id=i) for i in range(copies)]
    b = mcpd.Batch(ctx, [inst] * copies, params, order_mode=1, classes=1)
    est = torch.empty(b.total_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    ms = []
    with torch.cuda.stream(stream):
        for _ in range(3):
            b.run_async(est, se)
            st = b.collect()
            ms.append(st["kernel_ms"])
    info = [int(v) for v in b.info[:12]]
    b.close()
    return dict(ms=min(ms), draws=st["progress_units"], info=info)


def main(argv=None):
    ap = argparse.ArgumentParser(description="single-instance kernel against the batch kernel on the same draws")
    ap.add_argument("which", nargs="?", default="all", choices=("plan", "batch1", "batch128", "all"))
    which = ap.parse_args(argv).which
    import torch
    build.build()
    inst = synth.high_noise_config()
    stream = torch.cuda.Stream(0)
    ctx = mcpd.Context(0, stream=stream)
    out = {}
    if which in ("all", "plan"):
        out["plan"] = _plan(ctx, stream, inst)
    if which in ("all", "batch1"):
        out["batch1"] = _batch(ctx, stream, inst, 1)
    if which in ("all", "batch128"):
        out["batch128"] = _batch(ctx, stream, inst, 128)
    for v in out.values():
        v["ns_per_draw_per_pair"] = v["ms"] * 1e6 / v["draws"]
    print(json.dumps(out), flush=True)
    ctx.close()
    return out


if __name__ == "__main__":
    main()
