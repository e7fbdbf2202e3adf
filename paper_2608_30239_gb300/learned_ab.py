"""A/B of the learned initial marginals / scan weights against the paper's score weights.

  python -m paper_2608_30239_gb300.learned_ab [--train 4096] [--held 64] [--nu-floor 0.02]

1. Draw `train` instances shaped like the high-noise 1298 x 97 k = 6 workload (fp .10, fn .20,
   three positives, q = 3/1298; a new design and outcome seed each), estimate their marginals with
   the plain method (paper score weights, all-negative start, batched decode), compute features
   and train the MLP on the GPU.
2. On `held` further instances, decode with (a) the paper's score weights and the all-negative
   start, (b) paper weights and the learned initial marginals, (c) learned weights and learned
   initial marginals, all as one batched launch of P slots per instance and a 29.4-sweep horizon
   (the bench's B = 38146 at n = 1298).
3. Report per variant the largest per-clone standard error of each instance and the projected
   time to reach SE <= 0.005: the slot means are i.i.d., so SE scales as P^-1/2 and the decode time
   as P; projected time = (batch kernel time / instances) * (max SE / 0.005)^2 per instance.
4. With --direct, measure time-to-SE on the bench instance and the first `--direct-held` held-out
   instances: one decode per variant extended slot range by slot range until its largest SE is
   <= 0.005 (learned.time_to_se), reporting the summed kernel time and the wall time.
5. With --batched N, measure the batched form: the first N held-out instances decoded as one
   batch, extended until every instance's largest SE is <= 0.005 (learned.batched_time_to_se).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import synth

from . import learned, mcpd


def high_noise_like(i: int, base: int):
    return synth.make_instance(1298, 97, 6, 3, 0.10, 0.20, 3 / 1298, base + 2 * i, base + 2 * i + 1)


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--held", type=int, default=64)
    ap.add_argument("--slots", type=int, default=16384)
    ap.add_argument("--nu-floor", type=float, default=0.02)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--direct", action="store_true", help="also measure time-to-SE directly")
    ap.add_argument("--direct-held", type=int, default=4, help="held-out instances measured directly")
    ap.add_argument("--batched", type=int, default=0,
                    help="also measure the time for this many held-out instances, decoded as one batch, "
                         "to all reach SE <= 0.005 (learned.batched_time_to_se)")
    a = ap.parse_args(argv)
    ctx = mcpd.Context(0)
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    train = [high_noise_like(int(i), 100000) for i in rng.permutation(a.train)]
    held = [high_noise_like(i, 900000) for i in range(a.held)]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    p_hat, _, st_t = learned.plain_marginals(ctx, train, slots=1024, sweeps=10)
    t_targets = time.perf_counter() - t0
    seg = learned.segments(train)
    X = learned.features(ctx, train)
    tp = torch.tensor(np.clip(p_hat, 0.0, 1.0), dtype=torch.float32, device=X.device)
    tw = torch.tensor(learned.weight_target(p_hat, seg, mode="positive"), dtype=torch.float32, device=X.device)
    model = learned.MLP(ctx, seed=0)
    t0 = time.perf_counter()
    hist = model.fit(X, seg, tw, tp, epochs=a.epochs, batch_segments=64, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    hseg = learned.segments(held)
    Xh = learned.features(ctx, held)
    w, nu = learned.learned_inputs(model, Xh, hseg, nu_floor=a.nu_floor)
    variants = {"paper_weights_allneg": {}, "paper_weights_learned_nu": dict(init=nu),
                "learned_w_learned_nu": dict(weights=w, init=nu)}
    out = {"metric": "projected time to max per-clone SE <= 0.005 (learned vs paper weights)",
           "train_instances": a.train, "held_out": a.held, "slots": a.slots, "nu_floor": a.nu_floor,
           "nu_nonzero_per_instance": float((nu > 0).sum() / a.held),
           "seconds": {"generate": t_gen, "targets": t_targets, "train": t_train},
           "train_targets_kernel_ms": st_t["kernel_ms"], "loss_first_last": [hist[0], hist[-1]],
           "variants": {}}
    per_inst = {}
    for name, kw in variants.items():
        se, ms, st = _per_instance_max_se(ctx, held, a.slots, 29.4, 7, **kw)
        proj = (ms / 1000.0 / a.held) * (se / 0.005) ** 2
        per_inst[name] = proj
        out["variants"][name] = {
            "kernel_ms": ms, "max_se_over_instances": float(se.max()), "median_max_se": float(np.median(se)),
            "projected_s_median": float(np.median(proj)), "projected_s_batch": float(ms / 1000.0 * (se.max() / 0.005) ** 2),
            "mean_tau": st["sum_tau"] / max(1, st["reps_retained"]), "max_tau": st["max_tau"]}
    base = per_inst["paper_weights_allneg"]
    for name in variants:
        r = per_inst[name] / base
        out["variants"][name]["speedup_vs_paper_geomean"] = float(np.exp(-np.mean(np.log(r))))
        out["variants"][name]["instances_faster"] = int(np.sum(r < 1.0))
    if a.direct:
        out["direct"] = {}
        for label, inst in [("bench", synth.high_noise_config())] + \
                           [(f"held{i}", held[i]) for i in range(min(a.direct_held, a.held))]:
            Xb = learned.features(ctx, [inst])
            wb, nub = learned.learned_inputs(model, Xb, learned.segments([inst]), nu_floor=a.nu_floor)
            arms = {}
            for name, kw in (("paper_weights_allneg", {}), ("paper_weights_learned_nu", dict(init=nub)),
                             ("learned_w_learned_nu", dict(weights=wb, init=nub))):
                r = learned.time_to_se(ctx, inst, 0.005, 29.4, seed=7, **kw)
                arms[name] = {k: r[k] for k in ("kernel_ms", "wall_ms", "slots", "max_se", "met", "mean_tau")}
            base = arms["paper_weights_allneg"]["kernel_ms"]
            for v in arms.values():
                v["speedup_vs_paper"] = base / v["kernel_ms"]
            out["direct"][label] = arms
    if a.batched:
        sub = held[:a.batched]
        hs = learned.segments(sub)
        wb, nub = learned.learned_inputs(model, learned.features(ctx, sub), hs, nu_floor=a.nu_floor)
        arms = {}
        for name, kw in (("paper_weights_allneg", {}), ("paper_weights_learned_nu", dict(init=nub)),
                         ("learned_w_learned_nu", dict(weights=wb, init=nub))):
            arms[name] = learned.batched_time_to_se(ctx, sub, 0.005, 29.4, seed=7, **kw)
        base = arms["paper_weights_allneg"]["kernel_ms"]
        for v in arms.values():
            v["speedup_vs_paper"] = base / v["kernel_ms"]
        out["batched"] = {"instances": a.batched, "arms": arms}
    print(json.dumps(out), flush=True)
    ctx.close()
    return out


def _per_instance_max_se(ctx, instances, slots, sweeps, seed, weights=None, init=None):
    """Largest per-clone SE of each instance from one batched decode, its kernel ms and stats."""
    import torch
    seg = learned.segments(instances)
    params = []
    for i, inst in enumerate(instances):
        kw = dict(slots=slots, horizon=int(sweeps * inst.n), seed=seed + i, instance_id=i)
        if weights is not None:
            kw.update(scan=mcpd.MCPD_SCAN_CUSTOM, scan_weights=weights[seg[i]:seg[i + 1]])
        if init is not None:
            kw.update(init_marginals=init[seg[i]:seg[i + 1]])
        params.append(kw)
    b = mcpd.Batch(ctx, instances, params)
    est = torch.empty(b.total_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    b.run_async(est, se)
    st = b.collect()
    s = se.cpu().numpy()
    off = b.offsets
    b.close()
    return np.array([s[off[i]:off[i + 1]].max() for i in range(len(instances))]), st["kernel_ms"], st


if __name__ == "__main__":
    main()
