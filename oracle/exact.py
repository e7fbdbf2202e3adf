"""Exact posterior marginals and explicit transition matrices (test infrastructure only).

`posterior` enumerates all 2^n_a states of the pruned posterior of Knill's method (Section
"Knill's Method"):  pi_A(z) ∝ prod_{i in A} q^{z_i} (1-q)^{1-z_i} prod_j Pr{y_j | xi_j^A(z)},
with Pr{y=1|xi=1} = 1 - fn and Pr{y=1|xi=0} = fp.  `transition_matrices` builds the single-site
Gibbs matrices P_i(x, x') = 1{x_-i = x'_-i} p_i(x'_i | x_-i) and P_w = sum_i w_i P_i of the
Preliminaries, for checking pi P = pi (Proposition 1) on tiny designs.
"""
from __future__ import annotations

import numpy as np


def _incidence(inst, active):
    A = np.zeros((len(active), inst.m), dtype=np.int64)
    for a, i in enumerate(active):
        A[a, inst.clone_pools[inst.clone_ptr[i]:inst.clone_ptr[i + 1]]] = 1
    return A


def log_posterior_table(inst, active):
    """Unnormalised log pi_A(z) for every z in {0,1}^{n_a}; state index bit a = z_a."""
    na = len(active)
    if na > 24:
        raise ValueError("enumeration limited to n_a <= 24")
    states = np.arange(1 << na, dtype=np.int64)
    Z = ((states[:, None] >> np.arange(na)[None, :]) & 1).astype(np.int64)
    A = _incidence(inst, active)
    xi = (Z @ A) > 0                                            # [2^na, m]
    y = inst.y.astype(bool)[None, :]
    fp, fn, q = inst.fp, inst.fn, inst.q
    lik = np.where(xi, np.where(y, np.log1p(-fn), np.log(fn)),
                   np.where(y, np.log(fp), np.log1p(-fp))).sum(axis=1)
    k = Z.sum(axis=1)
    prior = k * np.log(q) + (na - k) * np.log1p(-q)
    return prior + lik, Z


def log_posterior(inst, active, Z):
    """Unnormalised log pi_A(z) for the states given as rows of Z ([S, n_a] 0/1), any n_a."""
    Z = np.asarray(Z, dtype=np.int64).reshape(-1, len(active))
    A = _incidence(inst, active)
    xi = (Z @ A) > 0
    y = inst.y.astype(bool)[None, :]
    fp, fn, q = inst.fp, inst.fn, inst.q
    lik = np.where(xi, np.where(y, np.log1p(-fn), np.log(fn)),
                   np.where(y, np.log(fp), np.log1p(-fp))).sum(axis=1)
    k = Z.sum(axis=1)
    return k * np.log(q) + (len(active) - k) * np.log1p(-q) + lik


def posterior(inst, active=None):
    """(pi over states, marginals p_j = E_pi[Z_j]) of the pruned posterior."""
    if active is None:
        active = np.arange(inst.n)
    lp, Z = log_posterior_table(inst, active)
    mx = lp.max()
    pi = np.exp(lp - mx)
    pi /= pi.sum()
    return pi, pi @ Z


def transition_matrices(cond_prob, na, weights):
    """P_i for every site from a full-conditional function cond_prob(state_index, i) -> p_i(1|x_-i),
    and P_w = sum_i w_i P_i."""
    S = 1 << na
    Ps = []
    for i in range(na):
        Pi = np.zeros((S, S))
        bit = 1 << i
        for s in range(S):
            p1 = cond_prob(s, i)
            Pi[s, s | bit] += p1
            Pi[s, s & ~bit] += 1.0 - p1
        Ps.append(Pi)
    Pw = sum(w * Pi for w, Pi in zip(weights, Ps))
    return Ps, Pw
