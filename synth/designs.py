"""Seeded random k-sets pooling designs and noisy pool outcomes.

The paper's synthetic instance (Section "Experimental Setup", synthetic data) is a Knill-type random
pooling design: every clone sits in the same number of pools, chosen at random; a few clones are
true positives; a pool's latent state is positive when it holds a positive clone; and the observed
outcome flips that state with the false-negative / false-positive rates.  The fixed instance the
paper used is not published, so these generators draw instances of the same shape from a seed.

Randomness comes from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter form, written
with numpy uint64 arithmetic so that every platform draws the same instance for the same seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class SplitMix64:
    """SplitMix64 stream: output i is mix64(seed + (i + 1) * golden_gamma)."""

    def __init__(self, seed: int):
        self.state = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(1, count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + idx * _GAMMA
            self.state = self.state + np.uint64(count) * _GAMMA
        return _mix64(z)

    def below(self, count: int, bound) -> np.ndarray:
        """`count` integers in [0, bound) (bound scalar or array): top 32 bits times bound, >> 32."""
        hi = self.u64(count) >> np.uint64(32)
        with np.errstate(over="ignore"):
            return ((hi * np.asarray(bound, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)

    def uniform(self, count: int) -> np.ndarray:
        """`count` doubles in [0, 1) with 53 random bits each."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Instance:
    """One pooling instance: clone->pool CSR, observed outcomes and the noise model."""
    n: int
    m: int
    clone_ptr: np.ndarray      # int32 [n + 1]
    clone_pools: np.ndarray    # int32 [nnz], each row strictly increasing
    y: np.ndarray              # uint8 [m], observed pool outcomes
    positives: np.ndarray      # int32, the true positive clones
    fp: float
    fn: float
    q: float
    seed: int = 0
    label: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.clone_ptr[-1])

    def pools_of(self, i: int) -> np.ndarray:
        return self.clone_pools[self.clone_ptr[i]:self.clone_ptr[i + 1]]

    def pool_sizes(self) -> np.ndarray:
        return np.bincount(self.clone_pools, minlength=self.m)


def _partial_shuffle(rng: SplitMix64, rows: int, universe: int, take: int) -> np.ndarray:
    """`rows` independent draws of `take` distinct items of range(universe) (Fisher-Yates prefix)."""
    picks = np.empty((rows, take), dtype=np.int64)
    offs = np.empty((rows, take), dtype=np.int64)
    for s in range(take):
        offs[:, s] = s + rng.below(rows, universe - s)
    for r in range(rows):
        perm = list(range(universe)) if universe <= 4 * take else None
        if perm is not None:
            for s in range(take):
                j = offs[r, s]
                perm[s], perm[j] = perm[j], perm[s]
            picks[r] = perm[:take]
        else:  # sparse Fisher-Yates: only swapped positions are stored
            swapped = {}
            for s in range(take):
                j = int(offs[r, s])
                vs, vj = swapped.get(s, s), swapped.get(j, j)
                swapped[s], swapped[j] = vj, vs
                picks[r, s] = vj
    return picks


def kset_design(n: int, m: int, deg: int, seed: int):
    """Random k-sets design: each clone joins `deg` distinct pools drawn uniformly."""
    if deg > m:
        raise ValueError("deg > m")
    rng = SplitMix64(seed)
    picks = np.sort(_partial_shuffle(rng, n, m, deg), axis=1)
    clone_ptr = np.arange(0, (n + 1) * deg, deg, dtype=np.int32)
    return clone_ptr, picks.reshape(-1).astype(np.int32)


def tapestry_like_design(n: int, m: int, deg: int, seed: int):
    """Regular design, a stand-in for the shape of the Tapestry designs: each clone sits in `deg`
    distinct pools, and the pool sizes differ by at most one (n deg / m each when m divides n deg).
    Clone-slots are dealt to the pools round robin in a shuffled order; a clone dealt the same pool
    twice swaps that entry with a randomly chosen entry of another clone (a swap keeps every pool's
    size), until no clone repeats a pool."""
    if deg > m:
        raise ValueError("deg > m")
    rng = SplitMix64(seed)
    order = np.argsort(rng.u64(n * deg), kind="stable")
    rows = (np.arange(n * deg, dtype=np.int64) % m)[order].reshape(n, deg)
    for i in range(n):
        for a in range(deg):
            for _ in range(1 << 20):
                if np.count_nonzero(rows[i] == rows[i, a]) == 1:
                    break
                j, b = (int(v) for v in rng.below(2, np.array([n, deg], dtype=np.uint64)))
                x, y = rows[i, a], rows[j, b]
                if j != i and y not in rows[i] and x not in rows[j]:
                    rows[i, a], rows[j, b] = y, x
            else:
                raise RuntimeError("no regular design found")
    clone_ptr = np.arange(0, (n + 1) * deg, deg, dtype=np.int32)
    return clone_ptr, np.sort(rows, axis=1).astype(np.int32).reshape(-1)


def mixed_degree_design(n: int, m: int, deg_lo: int, deg_hi: int, seed: int):
    """Each clone draws its own number of pools uniformly from [deg_lo, deg_hi], then that many
    distinct pools uniformly (rows of different lengths)."""
    if deg_hi > m or deg_lo < 1 or deg_lo > deg_hi:
        raise ValueError("need 1 <= deg_lo <= deg_hi <= m")
    rng = SplitMix64(seed)
    degs = deg_lo + rng.below(n, deg_hi - deg_lo + 1).astype(np.int64)
    picks = _partial_shuffle(rng, n, m, deg_hi)
    rows = [np.sort(picks[i, :degs[i]]) for i in range(n)]
    clone_ptr = np.zeros(n + 1, dtype=np.int32)
    clone_ptr[1:] = np.cumsum(degs)
    return clone_ptr, np.concatenate(rows).astype(np.int32)


def draw_outcomes(n: int, m: int, clone_ptr, clone_pools, n_pos: int, fp: float, fn: float,
                  seed: int):
    """Pick `n_pos` true positives uniformly, then y_j ~ Bern(1-fn) if pool j holds one, else
    Bern(fp)."""
    rng = SplitMix64(seed)
    positives = np.sort(_partial_shuffle(rng, 1, n, n_pos)[0]).astype(np.int32)
    xi = np.zeros(m, dtype=bool)
    for i in positives:
        xi[clone_pools[clone_ptr[i]:clone_ptr[i + 1]]] = True
    u = rng.uniform(m)
    y = np.where(xi, u < (1.0 - fn), u < fp).astype(np.uint8)
    return positives, y


def make_instance(n, m, deg, n_pos, fp, fn, q, design_seed, outcome_seed, label=""):
    clone_ptr, clone_pools = kset_design(n, m, deg, design_seed)
    positives, y = draw_outcomes(n, m, clone_ptr, clone_pools, n_pos, fp, fn, outcome_seed)
    return Instance(n=n, m=m, clone_ptr=clone_ptr, clone_pools=clone_pools, y=y,
                    positives=positives, fp=fp, fn=fn, q=q, seed=design_seed, label=label)


def make_mixed_instance(n, m, deg_lo, deg_hi, n_pos, fp, fn, q, design_seed, outcome_seed, label=""):
    """As `make_instance`, on a `mixed_degree_design`."""
    clone_ptr, clone_pools = mixed_degree_design(n, m, deg_lo, deg_hi, design_seed)
    positives, y = draw_outcomes(n, m, clone_ptr, clone_pools, n_pos, fp, fn, outcome_seed)
    return Instance(n=n, m=m, clone_ptr=clone_ptr, clone_pools=clone_pools, y=y,
                    positives=positives, fp=fp, fn=fn, q=q, seed=design_seed, label=label)


def make_tapestry_like_instance(n, m, deg, n_pos, fp, fn, q, design_seed, outcome_seed, label=""):
    """As `make_instance`, on a `tapestry_like_design` (the shape of the Tapestry designs)."""
    clone_ptr, clone_pools = tapestry_like_design(n, m, deg, design_seed)
    positives, y = draw_outcomes(n, m, clone_ptr, clone_pools, n_pos, fp, fn, outcome_seed)
    return Instance(n=n, m=m, clone_ptr=clone_ptr, clone_pools=clone_pools, y=y,
                    positives=positives, fp=fp, fn=fn, q=q, seed=design_seed, label=label)


def tiny_config(seed: int = 1) -> Instance:
    """20 clones, 8 pools, 3 pools per clone, 2 true positives, fp .02, fn .05, prior .01."""
    return make_instance(20, 8, 3, 2, 0.02, 0.05, 0.01, 1000 + seed, 2000 + seed,
                         label=f"tiny-20x8-k3-seed{seed}")


def paper_shaped_config(seed: int = 7) -> Instance:
    """1298 clones, 97 pools, 6 pools per clone, 3 true positives, fp .01, fn .05, q = 3/1298."""
    return make_instance(1298, 97, 6, 3, 0.01, 0.05, 3.0 / 1298.0, 5000 + seed, 6000 + seed,
                         label=f"lib-1298x97-k6-fp.01-fn.05-seed{seed}")


def high_noise_config(seed: int = 7) -> Instance:
    """The same 1298 x 97 k = 6 design as `paper_shaped_config`, outcomes at fp .10, fn .20."""
    return make_instance(1298, 97, 6, 3, 0.10, 0.20, 3.0 / 1298.0, 5000 + seed, 7000 + seed,
                         label=f"lib-1298x97-k6-fp.10-fn.20-seed{seed}")


def batched_configs(count: int = 512, seed: int = 11):
    """Uneven instances: n ~ U[200, 5000], m = round(n / 13), k ~ U{4..8}, 1-6 positives,
    fp ~ U[.005, .1], fn ~ U[.02, .25], q = positives / n."""
    rng = SplitMix64(seed)
    n_all = 200 + rng.below(count, 4801)
    k_all = 4 + rng.below(count, 5)
    pos_all = 1 + rng.below(count, 6)
    fp_all = 0.005 + rng.uniform(count) * (0.1 - 0.005)
    fn_all = 0.02 + rng.uniform(count) * (0.25 - 0.02)
    out = []
    for i in range(count):
        n = int(n_all[i])
        m = int(np.floor(n / 13.0 + 0.5))
        k = int(k_all[i])
        npos = int(pos_all[i])
        out.append(make_instance(n, m, k, npos, float(fp_all[i]), float(fn_all[i]), npos / n,
                                 100000 + 2 * i + seed * 7919, 100001 + 2 * i + seed * 7919,
                                 label=f"batch{i}-{n}x{m}-k{k}"))
    return out


def budget_horizon(budget_site_updates: float, slots: int) -> int:
    """Per-slot horizon B in progress units for a total budget of single-site updates: one
    progress unit of a coupled pair updates both chains, so B = floor(budget / (2 P))."""
    return int(budget_site_updates // (2 * slots))
