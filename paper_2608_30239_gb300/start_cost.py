"""Cost of random starts (Z_0 ~ prod Bernoulli(nu_i)) against the all-negative start.

  python -m paper_2608_30239_gb300.start_cost [--slots 262144] [--reps 3]

Decodes the high-noise 1298 x 97 k = 6 bench instance (horizon B = 38146, seed 7) with
(a) nu = 0 everywhere (no draws: the build without the random-start check),
(b) nu = 1e-4 on the 32, 164 and 656 highest-score clones (a draw per clone pair at every
    replication start, almost never a positive: the chains match (a), so the difference is the
    cost of drawing),
(c) nu = 0.3 on the 164 highest-score clones (draws and positive starts).
Reports the fastest of `reps` sampling-kernel times (CUDA events) per case, the replications and
their mean meeting time.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

import synth

from . import mcpd

CASES = (("delta0", 0.0, 0), ("tiny_nu_32", 1e-4, 32), ("tiny_nu_164", 1e-4, 164),
         ("tiny_nu_656", 1e-4, 656), ("nu0.3_164", 0.3, 164))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--slots", type=int, default=262144)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cases", default=",".join(c[0] for c in CASES))
    a = ap.parse_args(argv)
    import torch

    inst = synth.high_noise_config()
    info = mcpd.mcpd_inspect(inst, slots=8)
    order = info["active"][np.argsort(-info["w"], kind="stable")]    # clone ids by score weight
    ctx = mcpd.Context(0)
    out = {"workload": f"1298x97 k=6 high noise, {a.slots} slots, horizon 38146, seed 7", "cases": {}}
    wanted = set(a.cases.split(","))
    for label, val, count in CASES:
        if label not in wanted:
            continue
        kw = dict(slots=a.slots, horizon=38146, seed=7)
        if count:
            nu = np.zeros(inst.n)
            nu[order[:count]] = val
            kw["init_marginals"] = nu
        plan = mcpd.Plan(ctx, inst, **kw)
        est = torch.empty(plan.n_active, dtype=torch.float64, device="cuda:0")
        se = torch.empty_like(est)
        ms = []
        for _ in range(max(1, a.reps)):
            plan.run_async(est, se)
            st = plan.collect()
            ms.append(st["kernel_ms"])
        out["cases"][label] = dict(ms=min(ms), reps=st["reps_retained"],
                                   mean_tau=st["sum_tau"] / max(1, st["reps_retained"]))
        plan.close()
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
