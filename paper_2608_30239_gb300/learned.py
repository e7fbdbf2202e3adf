"""Learned scan weights and initial marginals for the coupled decoder (not in the paper).

The paper proves that any fixed positive scan weights leave the posterior invariant (Proposition 1)
and that the coupled estimator is unbiased from any initial distribution (Theorem 1).  This module
trains a small model to choose both from the observed design, with the library's own GPU kernels
(features, MLP forward/backward, Adam, heads; include/mcpd.h):

  targets  the method's own plain estimates p_hat on generated training instances (batched
           decode with the paper's score weights and an all-negative start);
  head 1   w = 0.5 softmax(o_1) + 0.5 / n, trained towards p_hat (1 - p_hat) + 0.01 normalised;
  head 2   nu = clamp(sigmoid(o_2)), trained towards p_hat (binary cross-entropy).

Only orchestration lives here (argument marshalling and the order of calls); every computation is
a library call.  `time_to_se` measures the decode time needed to bring the largest per-clone
standard error of an instance to a target, extending one fixed-budget decode slot range by slot
range until it gets there.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

from . import mcpd

_sigs_done = False


def _lib():
    global _sigs_done
    L = mcpd.lib()
    if not _sigs_done:
        P = C.c_void_p
        for name, res, args in (
            ("mcpd_mlp_num_params", C.c_int, []),
            ("mcpd_features_batch", C.c_int, [P, C.c_int32, P, P, P, P]),
            ("mcpd_mlp_forward", C.c_int, [P, C.c_int64, P, P, P]),
            ("mcpd_mlp_loss", C.c_int, [P, C.c_int32, P, P, P, P, P, P]),
            ("mcpd_mlp_backward", C.c_int, [P, C.c_int64, P, P, P, P, C.c_int64, P]),
            ("mcpd_mlp_backward_workspace", C.c_int64, [C.c_int64]),
            ("mcpd_mlp_adam", C.c_int, [P, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float,
                                        P, P, P, P, P]),
            ("mcpd_mlp_cast", C.c_int, [P, P, P]),
            ("mcpd_mlp_heads", C.c_int, [P, C.c_int32, P, P, P, P]),
        ):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _sigs_done = True
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def segments(instances) -> np.ndarray:
    return np.concatenate([[0], np.cumsum([inst.n for inst in instances])]).astype(np.int64)


def features(ctx, instances):
    """[sum n, 16] float32 device tensor of per-clone features, rows in instance order."""
    import torch
    keep = mcpd._Keep()
    n = len(instances)
    designs = (mcpd.mcpd_design * n)()
    ys = (C.c_void_p * n)()
    rates = np.zeros((n, 3))
    for i, inst in enumerate(instances):
        d, y = mcpd.make_design(inst, keep)
        designs[i] = d
        ys[i] = mcpd._ptr(y).value
        rates[i] = (inst.fp, inst.fn, inst.q)
    F = torch.empty((int(segments(instances)[-1]), 16), dtype=torch.float32, device=f"cuda:{ctx.device}")
    ctx.check(_lib().mcpd_features_batch(ctx.h, n, designs, ys, mcpd._ptr(rates), _p(F)),
              "mcpd_features_batch")
    return F


class MLP:
    """16-64-64-2 MLP: fp32 master parameters, bf16 copy used by the kernels, Adam state."""

    def __init__(self, ctx, seed: int = 0):
        import torch
        self.ctx = ctx
        self.n_params = int(_lib().mcpd_mlp_num_params())
        rng = np.random.default_rng(seed)
        theta = []
        for fan_out, fan_in in ((64, 16), (64, 64), (2, 64)):
            theta.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), fan_out * fan_in))
            theta.append(np.zeros(fan_out))
        theta = np.concatenate(theta).astype(np.float32)
        dev = f"cuda:{ctx.device}"
        self.master = torch.from_numpy(theta).to(dev)
        self.W = torch.empty(self.n_params, dtype=torch.int16, device=dev)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.grad = torch.zeros_like(self.master)
        self.step = 0
        self.cast()

    def cast(self):
        self.ctx.check(_lib().mcpd_mlp_cast(self.ctx.h, _p(self.master), _p(self.W)), "mcpd_mlp_cast")

    def forward(self, X):
        import torch
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        self.ctx.check(_lib().mcpd_mlp_forward(self.ctx.h, X.shape[0], _p(X), _p(self.W), _p(out)),
                       "mcpd_mlp_forward")
        return out

    def loss_grad(self, X, seg_dev, target_w, target_p):
        """Loss of the rows X (segments seg_dev) and its gradient in self.grad."""
        import torch
        out = self.forward(X)
        dout = torch.empty_like(out)
        nseg = seg_dev.numel() - 1
        lseg = torch.empty(nseg, dtype=torch.float64, device=X.device)
        self.ctx.check(_lib().mcpd_mlp_loss(self.ctx.h, nseg, _p(seg_dev), _p(out), _p(target_w),
                                            _p(target_p), _p(dout), _p(lseg)), "mcpd_mlp_loss")
        nwork = int(_lib().mcpd_mlp_backward_workspace(X.shape[0]))
        work = torch.empty(nwork, dtype=torch.float32, device=X.device)
        self.ctx.check(_lib().mcpd_mlp_backward(self.ctx.h, X.shape[0], _p(X), _p(self.W), _p(dout),
                                                _p(work), nwork, _p(self.grad)), "mcpd_mlp_backward")
        return float(lseg.cpu().numpy().sum()), out, dout

    def adam(self, lr=3e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step += 1
        self.ctx.check(_lib().mcpd_mlp_adam(self.ctx.h, self.step, lr, b1, b2, eps, _p(self.master),
                                            _p(self.m), _p(self.v), _p(self.grad), _p(self.W)),
                       "mcpd_mlp_adam")

    def heads(self, X, seg_dev):
        import torch
        out = self.forward(X)
        n = X.shape[0]
        w = torch.empty(n, dtype=torch.float64, device=X.device)
        nu = torch.empty_like(w)
        self.ctx.check(_lib().mcpd_mlp_heads(self.ctx.h, seg_dev.numel() - 1, _p(seg_dev), _p(out),
                                             _p(w), _p(nu)), "mcpd_mlp_heads")
        return w, nu

    def fit(self, X, seg, target_w, target_p, epochs=30, batch_segments=256, lr=3e-3, seed=0):
        """Adam over minibatches of whole instances: minibatch k is the contiguous block of
        instances [k * batch_segments, (k + 1) * batch_segments) (the caller draws the instances
        in random order), and each epoch visits the blocks in a fresh random order.  Returns the
        loss per epoch."""
        import torch
        dev = X.device
        seg = np.asarray(seg, np.int64)
        nseg = len(seg) - 1
        rng = np.random.default_rng(seed)
        blocks = [(a, min(nseg, a + batch_segments)) for a in range(0, nseg, batch_segments)]
        subs = [torch.from_numpy((seg[a:b + 1] - seg[a]).astype(np.int64)).to(dev) for a, b in blocks]
        hist = []
        for ep in range(epochs):
            tot = 0.0
            for k in rng.permutation(len(blocks)):
                a, b = blocks[k]
                r0, r1 = int(seg[a]), int(seg[b])
                loss, _, _ = self.loss_grad(X[r0:r1], subs[k], target_w[r0:r1], target_p[r0:r1])
                self.adam(lr)
                tot += loss * (b - a) / nseg
            hist.append(tot)
        return hist


def weight_target(p_hat: np.ndarray, seg: np.ndarray, floor: float = 0.01,
                  mode: str = "uncertainty") -> np.ndarray:
    """Per instance, normalised to sum 1: p_hat (1 - p_hat) + floor ("uncertainty": uncertain clones
    more often) or p_hat + floor ("positive": likely positives more often)."""
    pc = np.clip(p_hat, 0.0, 1.0)
    t = (pc * (1.0 - pc) if mode == "uncertainty" else pc) + floor
    out = np.empty_like(t)
    for s in range(len(seg) - 1):
        out[seg[s]:seg[s + 1]] = t[seg[s]:seg[s + 1]] / t[seg[s]:seg[s + 1]].sum()
    return out


def learned_inputs(model, X, seg, nu_floor: float = 1e-3):
    """(w, nu) host arrays for a decode: the heads' outputs, with nu_i < nu_floor set to 0.  Any
    initial marginals are admissible (Theorem 1), and zeros keep the start sparse: only clones
    with nu_i > 0 draw a starting bit."""
    import torch
    w, nu = model.heads(X, torch.from_numpy(np.asarray(seg, np.int64)).to(X.device))
    w = w.cpu().numpy()
    nu = nu.cpu().numpy()
    nu[nu < nu_floor] = 0.0
    return w, nu


def plain_marginals(ctx, instances, slots=256, sweeps=5, seed=1):
    """The method's own estimates p_hat (paper score weights, all-negative start), batched."""
    import torch
    params = [dict(slots=slots, horizon=sweeps * inst.n, seed=seed + i, instance_id=i % (1 << 24))
              for i, inst in enumerate(instances)]
    b = mcpd.Batch(ctx, instances, params, order_mode=0)
    est = torch.empty(b.total_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    b.run_async(est, se)
    st = b.collect()
    b.close()
    return est.cpu().numpy(), se.cpu().numpy(), st


def decode_max_se(ctx, instances, slots, sweeps, seed, weights=None, init=None, graph=False, lag_sweeps=0):
    """One batched decode of `instances` with P = slots and B = sweeps * n (lag-L pairs with
    L = lag_sweeps * n when lag_sweeps > 0); returns (max over instances of the largest per-clone
    SE, kernel ms, stats)."""
    import torch
    seg = segments(instances)
    params = []
    for i, inst in enumerate(instances):
        kw = dict(slots=slots, horizon=int(sweeps * inst.n), seed=seed + i, instance_id=i)
        if weights is not None:
            kw.update(scan=mcpd.MCPD_SCAN_CUSTOM, scan_weights=weights[seg[i]:seg[i + 1]])
        if init is not None:
            kw.update(init_marginals=init[seg[i]:seg[i + 1]])
        if lag_sweeps > 0:
            kw.update(lag=max(1, int(round(lag_sweeps * inst.n))))
        params.append(kw)
    t0 = time.perf_counter()
    b = mcpd.Batch(ctx, instances, params)
    est = torch.empty(b.total_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    b.run_async(est, se)
    st = b.collect()
    max_se = float(se.cpu().numpy().max())
    st["wall_ms"] = 1000.0 * (time.perf_counter() - t0)   # batch creation through the SE copy
    b.close()
    return max_se, st["kernel_ms"], st


def time_to_se(ctx, inst, target=0.005, sweeps=29.4, seed=7, weights=None, init=None, lag_sweeps=0,
               first_slots=1024, max_slots=1 << 26, plan_slots=524288):
    """Measured time to bring the largest per-clone SE of one instance to `target`.

    One fixed-budget decode (horizon B = sweeps * n progress units per slot, paper score weights
    unless `weights`, all-negative start unless `init`, lag-L pairs with L = lag_sweeps * n when
    lag_sweeps > 0) is extended slot range by slot range with mcpd_run_slots_async: each range adds
    the next global slot ids into the same integer N*_p buckets and the estimate is finalized over
    every slot so far, which is the same estimator as one decode over that many slots.  After each
    range the largest SE is read; the run stops at the first range that meets the target.  The next
    range's size comes from the SE's P^-1/2 law (slot means are i.i.d., Theorem 2): enough slots to
    reach the target if the law holds, at least `first_slots` and at most 8 times the slots so far.

    Returns the sampling kernels' summed CUDA-event time (`kernel_ms`), the wall time from plan
    creation through the copy of the SEs that met the target (`wall_ms`), the slots used, the final
    largest SE, whether it met the target, and the path [(slots so far, max SE, kernel ms so far)].
    The plan is shaped for `plan_slots` slots (the launch shape of the bench's decode); every range
    keeps its grid and trims its warps per block to whole rounds of the range."""
    import torch
    t0 = time.perf_counter()
    kw = dict(slots=plan_slots, horizon=int(sweeps * inst.n), seed=seed)
    if weights is not None:
        kw.update(scan=mcpd.MCPD_SCAN_CUSTOM, scan_weights=weights)
    if init is not None:
        kw.update(init_marginals=init)
    if lag_sweeps > 0:
        kw.update(lag=max(1, int(round(lag_sweeps * inst.n))))
    plan = mcpd.Plan(ctx, inst, **kw)
    est = torch.empty(plan.n_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    total, kernel_ms, path, add = 0, 0.0, [], int(first_slots)
    mean_tau_num = mean_tau_den = 0
    while True:
        plan.run_slots_async(add, est, se, accumulate=total > 0)
        st = plan.collect()
        total += add
        kernel_ms += st["kernel_ms"]
        mean_tau_num += st["sum_tau"]
        mean_tau_den += st["reps_retained"]
        mse = float(se.cpu().numpy().max())
        path.append((total, mse, kernel_ms))
        if mse <= target or total >= max_slots:
            break
        need = total * (mse / target) ** 2
        add = int(min(max(need * 1.02 - total, first_slots), 8 * total, max_slots - total))
        add = (add + 31) // 32 * 32
    wall_ms = 1000.0 * (time.perf_counter() - t0)
    plan.close()
    return dict(slots=total, max_se=mse, kernel_ms=kernel_ms, wall_ms=wall_ms, path=path,
                met=mse <= target, ranges=len(path), mean_tau=mean_tau_num / max(1, mean_tau_den))


def batched_time_to_se(ctx, instances, target=0.005, sweeps=29.4, seed=7, weights=None, init=None,
                       chunk_slots=131072, max_slots=1 << 26):
    """Measured time for a batch of instances to bring every instance's largest per-clone SE to
    `target`, decoded together: one batched decode with `chunk_slots` slots per instance (horizon
    `sweeps` sweeps of each instance's n), then extensions (mcpd_batch_extend_async) in which
    every instance not yet at the target runs its next `chunk_slots` slots, until all are there.
    Each instance's estimate is the same estimator over all its slots.  Returns the summed
    sampling-kernel time of the decode and its extensions, the wall time from batch creation
    through the last SE copy, the slots each instance used and its final largest SE."""
    import torch
    t0 = time.perf_counter()
    seg = segments(instances)
    params = []
    for i, inst in enumerate(instances):
        kw = dict(slots=chunk_slots, horizon=int(sweeps * inst.n), seed=seed + i, instance_id=i)
        if weights is not None:
            kw.update(scan=mcpd.MCPD_SCAN_CUSTOM, scan_weights=weights[seg[i]:seg[i + 1]])
        if init is not None:
            kw.update(init_marginals=init[seg[i]:seg[i + 1]])
        params.append(kw)
    b = mcpd.Batch(ctx, instances, params)
    est = torch.empty(b.total_active, dtype=torch.float64, device=f"cuda:{ctx.device}")
    se = torch.empty_like(est)
    off = b.offsets
    slots = np.full(len(instances), chunk_slots, np.int64)
    b.run_async(est, se)
    kernel_ms = b.collect()["kernel_ms"]
    rounds = 1
    while True:
        s = se.cpu().numpy()
        worst = np.array([s[off[i]:off[i + 1]].max() for i in range(len(instances))])
        todo = (worst > target).astype(np.int32)
        if not todo.any() or slots.max() + chunk_slots > max_slots:
            break
        b.extend_async(est, se, todo)
        kernel_ms += b.collect()["kernel_ms"]
        slots += chunk_slots * todo
        rounds += 1
    wall_ms = 1000.0 * (time.perf_counter() - t0)
    b.close()
    return dict(kernel_ms=kernel_ms, wall_ms=wall_ms, slots=slots.tolist(), max_se=worst.tolist(),
                met=bool((worst <= target).all()), launches=rounds)


def now() -> float:
    return time.perf_counter()
