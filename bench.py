#!/usr/bin/env python
"""Benchmark: coupled Gibbs site-updates/s of fixed-budget coupled score-weighted MCPD on GB300.

Workload: the 1298-clone x 97-pool k = 6 random k-sets design at high noise (fp .10, fn .20, three
true positives, q = 3/1298), 524288 logical slots per GPU, a budget of 4e10 single-site updates per
GPU (horizon B = 38146 progress units per slot), window l = n_a = 1298, k = 131.  One step is one
whole decode: every slot runs its coupled pairs to the horizon with refill (Algorithms 3-4), the
N*_p buckets are summed and theta_CT and its standard errors are finalized on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` counts single-site updates executed by the sampling kernel
(two per coupled draw, one for each replication's pre-lag draw) per second of device time with the
tables resident on the GPU; `e2e` is the same metric through mcpd_decode from host arrays to host
arrays.  The reference arm times the CPU oracle on the host's cores on a bounded slot sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled Gibbs site-updates/s"
UNIT = "site-updates/s"
SLOTS = 524288
BUDGET = 4e10
SEED = 20260
# DRAM bytes (read + written) per coupled draw of the sampling kernel on this workload, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the 87,552-slot case of this
# configuration (3.294e9 draws, 2.200 + 3.262 GB), scaled to a launch by its draws.  Taken for the
# current kernel revision; it is the accumulator events and flushes, not a per-step stream.
DRAM_BYTES_PER_DRAW = 1.6582


def workload_config(extra=None):
    cfg = {"workload": "MCPD high-noise 1298x97 k=6 fp=.10 fn=.20, 3 positives, q=3/1298; "
                       "524288 coupled-pair slots per GPU, budget 4e10 site-updates per GPU "
                       "(B=38146), window k=131 l=1298, score-weighted scan, all-negative start",
           "n_clones": 1298, "n_pools": 97, "pools_per_clone": 6, "slots_per_gpu": SLOTS,
           "budget_site_updates_per_gpu": BUDGET, "seed": SEED,
           "l2": "inputs smaller than L2 (tables are staged in shared memory); a 256 MiB buffer "
                 "is written between timed steps to flush L2"}
    if extra:
        cfg.update(extra)
    return cfg


def algorithmic_ops_per_progress_unit(deg: int) -> float:
    """Integer operations one coupled draw needs by the method's definition:
    half a Philox4x32-10 block (78 ops per block), the alias draw (4), per chain and per pool of the
    drawn site the 'no other positive' test and the (n+, n-) count (2 each), and per chain the
    64-bit threshold comparison (2)."""
    return 78 / 2 + 4 + 2 * (2 * deg) + 2 * 2


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mcpd_clocks_gpu{device_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it: the model name on x86, the implementer and part
    codes on Arm (where the kernel gives no model name); "unknown" elsewhere."""
    try:
        with open("/proc/cpuinfo") as f:
            fields = [line.split(":", 1) for line in f if ":" in line]
    except OSError:
        return "unknown"
    info = {}
    for k, v in fields:
        info.setdefault(k.strip(), v.strip())
    if "model name" in info:
        return info["model name"]
    if "CPU implementer" in info:
        return f"implementer {info['CPU implementer']} part {info.get('CPU part', '?')}"
    return "unknown"


def cpu_oracle_sample(seconds: float, steps_label: str = ""):
    """The oracle as it stands on the host's cores on a bounded sample of the workload's slots."""
    import oracle
    import synth
    inst = synth.high_noise_config()
    k, ell = oracle.window_defaults(inst.n, 1)
    B = synth.budget_horizon(BUDGET, SLOTS)
    cores = os.cpu_count() or 1
    M = oracle.Model(inst)
    run = oracle.coupled_run(k, ell, B, SEED)
    t0 = time.perf_counter()
    r = M.run_slots(run, 0, cores, cores)                      # calibration: one slot per core
    dt = time.perf_counter() - t0
    per_round = max(dt, 1e-3)
    rounds = max(1, int(seconds / per_round))
    n_slots = cores * rounds
    t0 = time.perf_counter()
    r = M.run_slots(oracle.coupled_run(k, ell, B, SEED, slot_offset=cores), 0, n_slots, cores)
    dt = time.perf_counter() - t0
    st = r["stats"]
    site_updates = 2 * st["draws"] - st["reps"]
    return {"value": site_updates / dt, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{n_slots} of the workload's {SLOTS} slots (slot ids {cores}..{cores + n_slots - 1}), "
                      f"{site_updates} site-updates in {dt:.2f} s with {cores} threads{steps_label}",
            "seconds": dt, "site_updates": site_updates}


def batched_leg(ctx, device, count=512, budget_slots=1024, budget_sweeps=20, seed=11, cap_sweeps=20,
                slot_candidates=(512, 1024, 2048), uncapped_limit_sweeps=None):
    """The uneven batch: `count` instances with n ~ U[200, 5000], m = round(n / 13), k ~ U{4..8},
    1-6 positives, fp ~ U[.005, .1], fn ~ U[.02, .25], q = positives / n.  Every instance gets the
    same budget in its own sweeps: `budget_slots` x `budget_sweeps` x n progress units, split into
    P slots of horizon budget_slots x budget_sweeps / P sweeps, with P (slots per instance) chosen by
    the autotuner among `slot_candidates` together with the launch shape (lanes per pair, warps per
    block; cached per GPU and shape).  One persistent launch per class (automatic classes: by
    degree, then by size, each on the build compiled for its degree), captured in one CUDA graph.  As in the paper's runs, pairs have a meeting cap of `cap_sweeps`
    sweeps (a pair unmet there is kept with its correction cut at the cap, and counted).  With
    `uncapped_limit_sweeps` the same batch is also decoded uncapped (the unbiased estimator), with a
    safety step limit of that many sweeps; its step-limit hits are reported (0 means the result is
    exactly the unbiased estimator)."""
    import torch

    import synth
    from paper_2608_30239_gb300 import autotune, mcpd
    stream = torch.cuda.Stream(device)         # graph capture needs a non-default stream
    ctx = mcpd.Context(device, stream=stream)
    t0 = time.perf_counter()
    insts = synth.batched_configs(count, seed=seed)
    name = torch.cuda.get_device_name(device)

    def params_for(P, capped=True):
        sweeps = budget_slots * budget_sweeps / P
        return [dict(slots=P, horizon=int(round(sweeps * inst.n)), seed=5000 + i, instance_id=i,
                     **(dict(meeting_cap=cap_sweeps * inst.n) if capped else
                        dict(step_limit=uncapped_limit_sweeps * inst.n, tau_audit=cap_sweeps * inst.n)))
                for i, inst in enumerate(insts)]

    with torch.cuda.stream(stream):
        P, batch, shape, slot_times, cached = autotune.tuned_slots(ctx, insts, params_for, slot_candidates, name)
    t_setup = time.perf_counter() - t0
    est = torch.empty(batch.total_active, dtype=torch.float64, device=f"cuda:{device}")
    se = torch.empty_like(est)
    batch.run_async(est, se)                     # warm-up with the chosen shape
    batch.collect(allow_step_limit=True)
    batch.capture_graph(est, se)
    ms = []
    for _ in range(2):
        batch.launch_graph()
        st = batch.collect(allow_step_limit=True)
        ms.append(st["kernel_ms"])
    out = {"instances": count, "budget_per_instance": f"{budget_slots} x {budget_sweeps} sweeps of its n",
           "slots_per_instance": P, "horizon_sweeps": budget_slots * budget_sweeps / P,
           "slots_autotune_ms": {str(k): v for k, v in slot_times.items()}, "autotune_cached": cached,
           "shape_lanes_warps": list(shape), "clones_total": int(sum(inst.n for inst in insts)),
           "setup_s": t_setup, "size_classes": batch.classes, "degree_build_classes": int(batch.info[12]),
           "graph_ms": statistics.mean(ms), "site_updates_per_step": st["site_updates"],
           "site_updates_per_s": st["site_updates"] / (statistics.mean(ms) / 1000.0),
           "replications_per_s": st["reps_retained"] / (statistics.mean(ms) / 1000.0),
           "meeting_cap_sweeps": cap_sweeps, "capped_pairs": st["tau_over_audit"],
           "pairs_attempted": st["reps_started"], "slots_total": count * P}
    batch.close()
    if uncapped_limit_sweeps:
        ub = mcpd.Batch(ctx, insts, params_for(P, capped=False), order_mode=1)
        ub.set_shape(shape[1], shape[0])
        with torch.cuda.stream(stream):
            ub.run_async(est, se)
            ust = ub.collect(allow_step_limit=True)
        out["uncapped"] = {"step_limit_sweeps": uncapped_limit_sweeps, "kernel_ms": ust["kernel_ms"],
                           "site_updates_per_s": ust["site_updates"] / (ust["kernel_ms"] / 1000.0),
                           "step_limit_hits": ust["step_limit_hits"], "status": ust["status"],
                           "pairs_with_tau_over_cap": ust["tau_over_audit"], "max_tau": ust["max_tau"],
                           "pairs_attempted": ust["reps_started"]}
        ub.close()
    stream.synchronize()
    ctx.close()
    return out


def library_leg(ctx, device, slots=262144, budget=1e10, seed=4242, steps=3):
    """The paper-shaped library workload (1298 x 97, 6 pools per clone, 3 positives, fp .01,
    fn .05, q = 3/1298) at its size: 262,144 slots and a budget of 1e10 single-site updates, decoded
    by the two methods it compares: coupled score-weighted pairs (Algorithms 3-4, B = 19073
    progress units per slot, one-sweep window) and uncoupled systematic scan (Algorithms 1-2, the
    same budget: B = 38146 draws per slot, b = 130, T = 1168).  Reports each one's site-updates/s
    (best of `steps` decodes), its largest per-clone SE, and the SE each would reach in one second
    of the sampling kernel (SE scales as P^-1/2)."""
    import torch

    import synth
    from paper_2608_30239_gb300 import mcpd
    inst = synth.paper_shaped_config()
    out = {"workload": "1298x97 k=6 fp=.01 fn=.05, 262144 slots, budget 1e10 site-updates; the library's "
                       "default one-sweep windows (coupled k = 131, l = 1298; uncoupled b = 130, T = 1168)"}
    for name, kw in (("coupled_score_weighted", dict(scan=mcpd.MCPD_SCAN_SCORE)),
                     ("uncoupled_systematic", dict(coupled=False, scan=mcpd.MCPD_SCAN_SYSTEMATIC))):
        plan = mcpd.Plan(ctx, inst, slots=slots, budget_site_updates=budget, seed=seed, **kw)
        est = torch.empty(plan.n_active, dtype=torch.float64, device=f"cuda:{device}")
        se = torch.empty_like(est)
        ms, st = [], None
        for _ in range(steps):
            plan.run_async(est, se)
            st = plan.collect()
            ms.append(st["kernel_ms"])
        best = min(ms)
        mse = float(se.max().item())
        out[name] = {"kernel_ms": best, "site_updates_per_s": st["site_updates"] / (best / 1000.0),
                     "max_se": mse, "max_se_at_1s_of_kernel": mse * (best / 1000.0) ** 0.5,
                     "replications": st["reps_retained"], "horizon": int(plan.horizon)}
        plan.close()
    return out


def learned_leg(ctx, device, train=4096, held=2):
    """Time to a largest per-clone SE of 0.005 on the bench instance (1298 x 97, high noise, a
    29.4-sweep horizon per slot, B = 38146), measured for every arm: one fixed-budget decode per arm
    extended slot range by slot range until it meets the target (learned.time_to_se), the time being
    the summed kernel time of its ranges (and the wall time from plan creation to the SE copy that
    met it).  Arms: the paper's score weights with the all-negative start (plain), paper weights
    with initial marginals from the MLP, learned weights and marginals, and the plain and
    learned-marginal arms with pairs of lag one sweep.  The MLP is trained on the GPU on `train`
    generated instances like the bench's (new design and outcome seeds each); `held` further
    held-out instances repeat the three lag-1 arms.  Arms under one second are run three times and
    the median kept (a launch that small is timed by its slowest pairs)."""
    import numpy as np
    import torch

    import synth
    from paper_2608_30239_gb300 import learned, learned_ab
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    tr = [learned_ab.high_noise_like(int(i), 100000) for i in rng.permutation(train)]
    p_hat, _, _ = learned.plain_marginals(ctx, tr, slots=1024, sweeps=10)
    seg = learned.segments(tr)
    X = learned.features(ctx, tr)
    model = learned.MLP(ctx, seed=0)
    model.fit(X, seg, torch.tensor(learned.weight_target(p_hat, seg, mode="positive"), dtype=torch.float32, device=X.device),
              torch.tensor(np.clip(p_hat, 0, 1), dtype=torch.float32, device=X.device), epochs=30, batch_segments=64)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"train_instances": train, "train_s": t_train, "target_max_se": 0.005, "horizon_sweeps": 29.4,
           "how": "measured: one decode per arm extended slot range by slot range (mcpd_run_slots_async) "
                  "until its largest per-clone SE <= 0.005; s_to_se = summed sampling-kernel time"}

    def arms_for(inst, lags):
        w, nu = learned.learned_inputs(model, learned.features(ctx, [inst]), learned.segments([inst]), nu_floor=0.02)
        arms = [("paper_weights_allneg", {}), ("paper_weights_learned_nu", dict(init=nu)),
                ("learned_w_learned_nu", dict(weights=w, init=nu))]
        if lags:
            arms += [("paper_weights_allneg_lag1sweep", dict(lag_sweeps=1.0)),
                     ("paper_weights_learned_nu_lag1sweep", dict(init=nu, lag_sweeps=1.0))]
        res = {}
        for name, kw in arms:
            runs = [learned.time_to_se(ctx, inst, 0.005, 29.4, seed=8, **kw)]
            if runs[0]["kernel_ms"] < 1000.0:
                runs += [learned.time_to_se(ctx, inst, 0.005, 29.4, seed=8, **kw) for _ in range(2)]
            r = runs[0]
            ms = statistics.median(x["kernel_ms"] for x in runs)
            res[name] = {"s_to_se_0.005": ms / 1000.0, "wall_s": statistics.median(x["wall_ms"] for x in runs) / 1000.0,
                         "slots": r["slots"], "max_se": r["max_se"], "met": r["met"], "ranges": r["ranges"],
                         "mean_tau": r["mean_tau"], "kernel_ms_runs": [x["kernel_ms"] for x in runs]}
        base = res["paper_weights_allneg"]["s_to_se_0.005"]
        for v in res.values():
            v["speedup_vs_plain"] = base / v["s_to_se_0.005"]
        return res

    out["bench_instance"] = arms_for(synth.high_noise_config(), True)
    out["held_out"] = [arms_for(learned_ab.high_noise_like(i, 900000), False) for i in range(held)]
    b = out["bench_instance"]
    out["speedup"] = b["paper_weights_learned_nu"]["speedup_vs_plain"]
    out["speedup_learned_w_nu"] = b["learned_w_learned_nu"]["speedup_vs_plain"]
    out["speedup_lag1sweep"] = b["paper_weights_allneg_lag1sweep"]["speedup_vs_plain"]
    out["speedup_learned_nu_lag1sweep"] = b["paper_weights_learned_nu_lag1sweep"]["speedup_vs_plain"]
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_oracle_sample(2.0)
    vals, times = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        s = cpu_oracle_sample(args.ref_seconds)
        vals.append(s["value"])
        times.append(s["seconds"])
    wall = time.perf_counter() - t_all
    value = sum(vals) / len(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "impl": "reference", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": f"each step a bounded slot sample of ~{args.ref_seconds:.0f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def auxiliary_leg(leg, *args):
    """Run one leg beside the main figure.  If it raises, the line carries the error in its place
    (and the main figure, already measured, is still printed)."""
    try:
        return leg(*args)
    except Exception as e:                  # reported in the JSON line, not hidden
        return {"error": f"{type(e).__name__}: {e}"[:500]}


def reduce_over_ranks(dist, device, total_s, su_step, reps_step, e2e_s):
    """Whole-job figures from each rank's own: the slowest rank's timed seconds and end-to-end
    seconds per step (MAX), and one step's site updates and retained replications summed over the
    ranks (SUM).  `dist` is None for a single process; `device` holds the reduced tensors."""
    if dist is None:
        return float(total_s), float(su_step), float(reps_step), float(e2e_s)
    import torch
    slow = torch.tensor([float(total_s), float(e2e_s)], dtype=torch.float64, device=device)
    dist.all_reduce(slow, op=dist.ReduceOp.MAX)
    work = torch.tensor([float(su_step), float(reps_step)], dtype=torch.float64, device=device)
    dist.all_reduce(work, op=dist.ReduceOp.SUM)
    return float(slow[0].item()), float(work[0].item()), float(work[1].item()), float(slow[1].item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-instance batch leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned time-to-SE leg")
    ap.add_argument("--no-library", action="store_true", help="skip the library-shaped two-method leg")
    ap.add_argument("--slots", type=int, default=SLOTS,
                    help="slots per GPU; the budget scales with it so the horizon B stays 38146 "
                         "(smaller cases are for profiling captures)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import synth
    from paper_2608_30239_gb300 import build as lib_build
    from paper_2608_30239_gb300 import mcpd

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    device = local_rank
    torch.cuda.set_device(device)
    lib_build.build()

    inst = synth.high_noise_config()
    slots = args.slots
    budget = BUDGET * slots / SLOTS
    offset = rank * slots
    ctx = mcpd.Context(device)
    plan = mcpd.Plan(ctx, inst, slots=slots, budget_site_updates=budget, seed=SEED,
                     slot_offset=offset)
    est = torch.empty(plan.n_active, dtype=torch.float64, device=f"cuda:{device}")
    se = torch.empty_like(est)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{device}")
    stream = torch.cuda.current_stream(device)

    for _ in range(args.warmup):
        plan.run_async(est, se)
        plan.collect()

    clocks = ClockSampler(device)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                       # L2 flush, outside the timed interval
        ev[i][0].record(stream)
        plan.run_async(est, se)
        ev[i][1].record(stream)
        stats.append(plan.collect())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()

    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1000.0
    su_step = stats[-1]["site_updates"]
    pu_step = stats[-1]["progress_units"]
    kernel_ms = statistics.mean(s["kernel_ms"] for s in stats)

    # end to end through the public host-array API: plan, upload, run, download, every step; the
    # bytes are the library's own count of what it copied (tables up; counters, estimates and
    # standard errors down)
    e2e_times = []
    h2d = d2h = 0
    for i in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ctx.decode(inst, slots=slots, budget_site_updates=budget, seed=SEED, slot_offset=offset)
        e2e_times.append(time.perf_counter() - t0)
        assert out["status"] == 0
        h2d, d2h = out["stats"]["h2d_bytes"], out["stats"]["d2h_bytes"]
    total_s, su_all_step, reps_all_step, e2e_s = reduce_over_ranks(
        dist, f"cuda:{device}", total_s, su_step, stats[-1]["reps_retained"], statistics.mean(e2e_times))
    value = su_all_step * args.steps / total_s
    e2e_val = su_all_step / e2e_s

    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(device)
    sm_count = props.multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
    peak_ops = 128.0 * sm_count * max_mhz * 1e6       # 4 schedulers x 32 lanes issue per clock
    ops = algorithmic_ops_per_progress_unit(6) * pu_step
    achieved = ops / (kernel_ms / 1000.0)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tops/s", "frac": achieved / peak_ops,
                "traffic": DRAM_BYTES_PER_DRAW * pu_step, "traffic_unit": "bytes per launch",
                "note": f"issue-slot peak = 128 lane-ops/clk/SM x {sm_count} SMs x {max_mhz:.0f} MHz "
                        f"({peak_kind} max clock); algorithmic ops = "
                        f"{algorithmic_ops_per_progress_unit(6):.0f} per coupled draw"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": workload_config({"parallelism": f"slot shards x{world}",
                                       "slots_per_gpu": slots, "budget_site_updates_per_gpu": budget,
                                       "progress_units_per_step": pu_step,
                                       "site_updates_per_step": su_step,
                                       "replications_per_step": stats[-1]["reps_retained"],
                                       "estimators_per_s": reps_all_step * args.steps / total_s,
                                       "pairs_kernel_ms": kernel_ms,
                                       "max_se": float(se.max().item()),
                                       "wall_s_timed": wall}),
            "roofline": roofline,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "seconds_per_step": e2e_s},
            "gpu_launches": 2 * args.steps,
            "clocks": clk}
    if rank == 0 and not args.no_batched:
        line["batched"] = auxiliary_leg(batched_leg, ctx, device, 512, 1024, 20, 11, 20, (512, 1024, 2048),
                                        10000)
    if rank == 0 and not args.no_learned:
        line["time_to_se"] = auxiliary_leg(learned_leg, ctx, device)
    if rank == 0 and not args.no_library:
        line["library_config"] = auxiliary_leg(library_leg, ctx, device)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = auxiliary_leg(cpu_oracle_sample, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
