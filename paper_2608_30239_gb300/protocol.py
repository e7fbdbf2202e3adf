"""The five-method comparison on a synthetic instance (the protocol of the paper's experiments,
Section "Experimental Setup", on a generated stand-in for its unpublished instance).

  python -m paper_2608_30239_gb300.protocol [--noise 0.10,0.10] [--sweeps 1,3,5,10,20] [--slots 1000000]

Defaults follow the paper's synthetic instance: 1298 clones x 97 pools, 3 pools per clone, three
true positives, prior q = 2.6 / n, pruned to 333 clones; 1,000,000 coupled slots, 2,000,000
uncoupled chains, a 2,000,000-chain reference.

Methods, at an estimator length of s sweeps (M = s n_a single-site updates, b = round(0.1 M)):
  SS   systematic scan, uncoupled: discard b updates, average the next M - b (Algorithm 1);
  RU   uniform random scan, uncoupled (Algorithm 1);
  SW   score-weighted random scan, uncoupled (Algorithm 2);
  cRU  uniform random scan, coupled pairs, k = b + 1, l = M (Algorithms 3-4);
  cSW  score-weighted random scan, coupled pairs (Algorithms 3-4);
  cSW-nr  cSW without slot refill (the ablation of Section "Slot refill ablation"): a horizon of
       zero progress units, so every slot keeps its first pair and runs no other.
Every slot but those of cSW-nr has a horizon of 20 sweeps.  The uncoupled methods hold twice as many slots as the
coupled ones (each coupled slot holds two chains), so both hold the same number of chain states.
The reference vector is a long systematic-scan run (burn-in and sampling lengths in sweeps).
Scores are the mean absolute error over the retained clones and over the reference's ten largest.
As in the paper's runs, the coupled runs impose a 20-sweep meeting cap (a pair unmet at the cap is
kept with its correction cut there); the cap-hit rate is the share of the pairs attempted that
reached it.  With --uncapped the runs are unbiased and the rate counts the kept pairs whose
meeting time exceeded the cap.
--lag L runs the coupled methods with lag-L pairs (L pre-lag updates; the cap must be >= L).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import synth

from . import mcpd


def _decode(ctx, inst, **kw):
    import torch
    plan = mcpd.Plan(ctx, inst, **kw)
    est = torch.empty(plan.n_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    plan.run_async(est, se)
    st = plan.collect(allow_step_limit=True)
    out = est.cpu().numpy(), plan.active.copy(), st
    plan.close()
    return out


def _summary(rows):
    """Mean and standard error over executions of each (sweeps, method) cell."""
    cells = {}
    for r in rows:
        cells.setdefault((r["sweeps"], r["method"]), []).append(r)
    out = []
    for (s, m), rs in cells.items():
        d = {"sweeps": s, "method": m, "n": len(rs)}
        for key in ("mae_all", "mae_top10", "kernel_ms"):
            v = np.array([r[key] for r in rs], dtype=float)
            d[key] = float(v.mean())
            d[key + "_se"] = float(v.std(ddof=1) / np.sqrt(len(v))) if len(v) > 1 else None
        out.append(d)
    return out


def round_half_even(x: float) -> int:
    return int(np.round(x))


METHODS = {
    "SS": dict(coupled=False, scan=mcpd.MCPD_SCAN_SYSTEMATIC),
    "RU": dict(coupled=False, scan=mcpd.MCPD_SCAN_UNIFORM),
    "SW": dict(coupled=False, scan=mcpd.MCPD_SCAN_SCORE),
    "cRU": dict(coupled=True, scan=mcpd.MCPD_SCAN_UNIFORM),
    "cSW": dict(coupled=True, scan=mcpd.MCPD_SCAN_SCORE),
    "cSW-nr": dict(coupled=True, scan=mcpd.MCPD_SCAN_SCORE, horizon=0),
}


def cell_params(method, sweeps, n_active, slots, horizon_sweeps=20, cap_sweeps=20, uncapped=False, lag=1):
    """Decode parameters of one cell (method at an estimator length of `sweeps` sweeps), the
    paper's recipe (Section "Experimental Setup"; Table S1): M = s n_a, b = round(0.1 M); uncoupled
    methods discard b updates and average M - b over 2 `slots` chains; coupled methods use k = b + 1,
    l = M over `slots` pairs with a meeting cap of `cap_sweeps` sweeps (audited, not imposed, when
    `uncapped`); every slot has a horizon of `horizon_sweeps` sweeps except the no-refill ablation."""
    kw = dict(METHODS[method])
    M = sweeps * n_active
    b = round_half_even(0.1 * M)
    if kw["coupled"]:
        cap = cap_sweeps * n_active
        kw.update(k=b + 1, ell=M, slots=slots, tau_audit=cap, lag=lag)
        if not uncapped:
            kw["meeting_cap"] = cap
    else:
        kw.update(burn=b, length=M - b, slots=2 * slots)
    kw.setdefault("horizon", horizon_sweeps * n_active)
    kw["n_active"] = n_active
    return kw


def top_clones(ref, count=10):
    """The reference's `count` largest marginals (ties to the lower position)."""
    return np.argsort(-np.asarray(ref), kind="stable")[:count]


def scores(est, ref, top):
    """(all-clone MAE, top-10 MAE): mean |est - ref| over every retained clone and over `top`."""
    est, ref = np.asarray(est, float), np.asarray(ref, float)
    return float(np.mean(np.abs(est - ref))), float(np.mean(np.abs(est[top] - ref[top])))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1298)
    ap.add_argument("--m", type=int, default=97)
    ap.add_argument("--deg", type=int, default=3, help="pools per clone (the paper's synthetic instance: 3)")
    ap.add_argument("--positives", type=int, default=3)
    ap.add_argument("--prior", type=float, default=-1.0,
                    help="prior q (default 2.6 / n, the paper's synthetic runs; 0: positives / n)")
    ap.add_argument("--noise", default="0.10,0.10", help="fn,fp")
    ap.add_argument("--n-active", type=int, default=333)
    ap.add_argument("--sweeps", default="1,3,5,10,20")
    ap.add_argument("--horizon-sweeps", type=int, default=20)
    ap.add_argument("--slots", type=int, default=1000000, help="coupled slots (uncoupled: twice as many)")
    ap.add_argument("--ref-burn", type=int, default=1000, help="reference burn-in, sweeps")
    ap.add_argument("--ref-sweeps", type=int, default=10000, help="reference sampling length, sweeps")
    ap.add_argument("--ref-chains", type=int, default=2000000)
    ap.add_argument("--seed", type=int, default=20260)
    ap.add_argument("--cap-sweeps", type=int, default=20, help="meeting cap, sweeps")
    ap.add_argument("--uncapped", action="store_true", help="audit the cap without imposing it")
    ap.add_argument("--lag", type=int, default=1, help="lag of the coupled pairs")
    ap.add_argument("--methods", default="SS,RU,SW,cRU,cSW,cSW-nr", help="subset of the methods")
    ap.add_argument("--executions", type=int, default=1,
                    help="independent executions per cell (new seeds), summarised as mean and SE")
    a = ap.parse_args(argv)
    fn, fp = (float(v) for v in a.noise.split(","))
    q = a.prior if a.prior > 0 else (2.6 / a.n if a.prior < 0 else a.positives / a.n)
    inst = synth.make_instance(a.n, a.m, a.deg, a.positives, fp, fn, q, 5007, 9007)
    ctx = mcpd.Context(0)
    t0 = time.perf_counter()
    ref, active, st_ref = _decode(ctx, inst, n_active=a.n_active, coupled=False, scan=mcpd.MCPD_SCAN_SYSTEMATIC,
                                  burn=a.ref_burn * a.n_active, length=a.ref_sweeps * a.n_active,
                                  horizon=(a.ref_burn + a.ref_sweeps) * a.n_active, slots=a.ref_chains,
                                  seed=a.seed + 1)
    t_ref = time.perf_counter() - t0
    top = top_clones(ref)
    methods = [m for m in a.methods.split(",")]
    sweeps = [int(v) for v in a.sweeps.split(",")]
    rows = []
    for e in range(a.executions):
        for si, s in enumerate(sweeps):
            for ci, name in enumerate(methods):
                kw = METHODS[name]
                kw2 = cell_params(name, s, a.n_active, a.slots, a.horizon_sweeps, a.cap_sweeps, a.uncapped, a.lag)
                t1 = time.perf_counter()
                # one seed per (length, method) cell, shifted for each further execution
                seed = a.seed + 100 * s + si * len(methods) + ci + 1000003 * e
                est, act, st = _decode(ctx, inst, seed=seed, **kw2)
                assert np.array_equal(act, active)
                mae_all, mae_top = scores(est, ref, top)
                rows.append({"execution": e, "sweeps": s, "method": name, "mae_all": mae_all,
                             "mae_top10": mae_top,
                             "site_updates": st["site_updates"], "kernel_ms": st["kernel_ms"],
                             "step_limit_hits": st["step_limit_hits"], "reps_retained": st["reps_retained"],
                             "mean_tau_sweeps": (st["sum_tau"] / max(1, st["reps_retained"]) / a.n_active) if kw["coupled"] else None,
                             "max_tau_sweeps": (st["max_tau"] / a.n_active) if kw["coupled"] else None,
                             "reps_started": st["reps_started"],
                             "cap_hits": st["tau_over_audit"] if kw["coupled"] else None,
                             "cap_hit_rate": (st["tau_over_audit"] / max(1, st["reps_started"])) if kw["coupled"] else None,
                             "seconds": time.perf_counter() - t1})
    out = {"instance": dict(n=a.n, m=a.m, deg=a.deg, positives=a.positives, fn=fn, fp=fp, prior=q,
                            n_active=a.n_active),
           "reference": dict(burn_sweeps=a.ref_burn, sweeps=a.ref_sweeps, chains=a.ref_chains, seconds=t_ref,
                             site_updates=st_ref["site_updates"], top10=[int(active[i]) for i in top]),
           "slots_coupled": a.slots, "slots_uncoupled": 2 * a.slots, "horizon_sweeps": a.horizon_sweeps,
           "meeting_cap_sweeps": None if a.uncapped else a.cap_sweeps, "lag": a.lag,
           "executions": a.executions, "rows": rows, "summary": _summary(rows)}
    print(json.dumps(out), flush=True)
    ctx.close()
    return out


if __name__ == "__main__":
    main()
