"""CPU reference of the learned scan-weight / initial-marginal model (test infrastructure only).

Not part of the paper's method: the paper proves (Proposition 1, Theorem 1) that any fixed
positive scan weights w and any initial distribution nu keep pi invariant and H_{k:l} unbiased.
The library learns w and nu from per-clone features; this module restates, in plain fp64 numpy,
what its GPU kernels compute, so that their features, outputs and gradients can be checked:

  features(inst)        16 per-clone features of the design and outcomes (definitions below)
  forward(X, params)    MLP 16-64-64-2 with ReLU, weights rounded to bf16 by the caller
  heads(O, seg)         w = (1 - a) softmax_instance(o_1) + a / n,  nu = clamp(sigmoid(o_2))
  loss_and_grad(...)    cross-entropy of softmax(o_1) to a target distribution per instance plus
                        binary cross-entropy of sigmoid(o_2) to target marginals, and its gradient

The gradient is pinned by central finite differences in tests/test_learned_oracle.py.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 16
HIDDEN = 64
N_OUT = 2
ALPHA_W = 0.5
NU_MIN, NU_MAX = 1e-6, 1.0 - 1e-6
LAYER_SHAPES = [(HIDDEN, N_FEATURES), (HIDDEN, HIDDEN), (N_OUT, HIDDEN)]


def n_params() -> int:
    return sum(o * i + o for o, i in LAYER_SHAPES)


def unpack(theta: np.ndarray):
    """Flat parameter vector -> [(W1, b1), (W2, b2), (W3, b3)] (weights row-major [out][in])."""
    out, off = [], 0
    for o, i in LAYER_SHAPES:
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> np.uint64(16)) & np.uint64(1)
    r = ((f + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(inst) -> np.ndarray:
    """16 features per clone (float64).  With deg_i = |P(i)|, npos_i the positive pools of i,
    d_j the pool sizes, dbar = nnz / m, allpos_i = 1{npos_i = deg_i > 0}, ap_j the number of
    all-positive clones in pool j and NAP their total:
      0 deg/8  1 npos/8  2 nneg/8  3 npos/deg  4 eta/10 with eta = lambda + npos a+ + nneg a-
      5 mean_{j in P(i)} d_j / dbar   6 mean over positive pools of d_j / dbar (0 if none)
      7 allpos   8 min over positive pools of ap_j / 10 (0 if none)
      9 mean over positive pools of 1 / max(ap_j, 1) (0 if none)
      10 #positive pools with allpos_i = 1 and ap_j = 1 (i the only all-positive member) / 8
      11 #positive pools with ap_j = 0 / 8   12 NAP / 100   13 lambda/10  14 a+/10  15 a-/10."""
    n, m = inst.n, inst.m
    ptr, pools, y = inst.clone_ptr, inst.clone_pools, inst.y.astype(np.int64)
    a_pos = np.log(1.0 - inst.fn) - np.log(inst.fp)
    a_neg = np.log(inst.fn) - np.log(1.0 - inst.fp)
    lam = np.log(inst.q) - np.log(1.0 - inst.q)
    d = np.bincount(pools, minlength=m).astype(np.float64)
    dbar = len(pools) / m if m else 1.0
    deg = np.diff(ptr).astype(np.int64)
    npos = np.array([y[pools[ptr[i]:ptr[i + 1]]].sum() for i in range(n)], dtype=np.int64)
    allpos = ((npos == deg) & (deg > 0)).astype(np.int64)
    ap = np.zeros(m, dtype=np.int64)
    for i in range(n):
        if allpos[i]:
            ap[pools[ptr[i]:ptr[i + 1]]] += 1
    NAP = allpos.sum()
    F = np.zeros((n, N_FEATURES))
    for i in range(n):
        P = pools[ptr[i]:ptr[i + 1]]
        pos = P[y[P] == 1]
        nneg = deg[i] - npos[i]
        F[i, 0] = deg[i] / 8.0
        F[i, 1] = npos[i] / 8.0
        F[i, 2] = nneg / 8.0
        F[i, 3] = npos[i] / max(deg[i], 1)
        F[i, 4] = (lam + npos[i] * a_pos + nneg * a_neg) / 10.0
        F[i, 5] = (d[P].mean() / dbar) if len(P) else 0.0
        F[i, 6] = (d[pos].mean() / dbar) if len(pos) else 0.0
        F[i, 7] = allpos[i]
        F[i, 8] = (ap[pos].min() / 10.0) if len(pos) else 0.0
        F[i, 9] = (1.0 / np.maximum(ap[pos], 1)).mean() if len(pos) else 0.0
        F[i, 10] = (np.sum(ap[pos] == 1) if allpos[i] else 0) / 8.0
        F[i, 11] = np.sum(ap[pos] == 0) / 8.0
        F[i, 12] = NAP / 100.0
        F[i, 13] = lam / 10.0
        F[i, 14] = a_pos / 10.0
        F[i, 15] = a_neg / 10.0
    return F


def forward(X: np.ndarray, layers):
    """Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2, H2 = relu(Z2), O = H2 W3^T + b3."""
    (W1, b1), (W2, b2), (W3, b3) = layers
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    O = H2 @ W3.T + b3
    return Z1, H1, Z2, H2, O


def heads(O: np.ndarray, seg: np.ndarray):
    """Scan weights per instance (segment s = rows seg[s]..seg[s+1]) and initial marginals."""
    w = np.zeros(len(O))
    for s in range(len(seg) - 1):
        o = O[seg[s]:seg[s + 1], 0]
        e = np.exp(o - o.max())
        n = len(o)
        w[seg[s]:seg[s + 1]] = (1.0 - ALPHA_W) * e / e.sum() + ALPHA_W / n
    nu = np.clip(1.0 / (1.0 + np.exp(-O[:, 1])), NU_MIN, NU_MAX)
    return w, nu


def loss_and_dO(O: np.ndarray, seg: np.ndarray, target_w: np.ndarray, target_p: np.ndarray):
    """Mean over instances of [ -sum_i t_i log softmax(o_1)_i  +  mean_i BCE(sigmoid(o_2,i), p_i) ]
    and its gradient with respect to O."""
    n_inst = len(seg) - 1
    dO = np.zeros_like(O)
    total = 0.0
    for s in range(n_inst):
        a, b = seg[s], seg[s + 1]
        o1 = O[a:b, 0]
        mx = o1.max()
        lse = mx + np.log(np.exp(o1 - mx).sum())
        sm = np.exp(o1 - lse)
        t = target_w[a:b]
        ce = -(t * (o1 - lse)).sum()
        dO[a:b, 0] = (sm * t.sum() - t) / n_inst
        z = O[a:b, 1]
        p = target_p[a:b]
        bce = np.mean(np.logaddexp(0.0, z) - p * z)     # softplus(z) - p z
        sig = 1.0 / (1.0 + np.exp(-z))
        dO[a:b, 1] = (sig - p) / (b - a) / n_inst
        total += (ce + bce) / n_inst
    return total, dO


def backward(X, layers, cache, dO):
    """Gradients of sum(dO * O) with respect to every weight and bias (same layout as unpack)."""
    (W1, b1), (W2, b2), (W3, b3) = layers
    Z1, H1, Z2, H2, O = cache
    gW3 = dO.T @ H2
    gb3 = dO.sum(axis=0)
    dH2 = dO @ W3
    dZ2 = dH2 * (Z2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def weight_target(p_hat: np.ndarray, seg: np.ndarray, floor: float = 0.01) -> np.ndarray:
    """Target scan distribution per instance: proportional to p(1-p) + floor, normalised, so that
    clones whose marginal is uncertain are updated more often."""
    t = np.zeros(len(p_hat))
    pc = np.clip(p_hat, 0.0, 1.0)
    for s in range(len(seg) - 1):
        v = pc[seg[s]:seg[s + 1]] * (1.0 - pc[seg[s]:seg[s + 1]]) + floor
        t[seg[s]:seg[s + 1]] = v / v.sum()
    return t
