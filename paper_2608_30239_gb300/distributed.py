"""Exact combination of per-rank N*_p bucket sums across processes.

Slots are independent and keyed by their global id, so ranks run disjoint slot ranges
(slot_offset) and the only exchange is an integer sum of the buckets: S1 (int64), S2 (128-bit as
two uint64 words) and the slot counts.  S2 is split into four 32-bit limbs carried in int64 so the
sum is exact for any realistic world size, then recombined with carries.
"""
from __future__ import annotations

import numpy as np


def _limbs(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    m = np.uint64(0xFFFFFFFF)
    return np.stack([(lo & m), (lo >> np.uint64(32)), (hi & m), (hi >> np.uint64(32))]).astype(np.int64)


def _unlimb(l: np.ndarray):
    """Carry-propagate four int64 limb sums (each < 2^63) back into (lo, hi) uint64 words."""
    out = []
    carry = np.zeros(l.shape[1:], dtype=object)
    words = []
    for i in range(4):
        v = l[i].astype(object) + carry
        words.append(v % (1 << 32))
        carry = v // (1 << 32)
    lo = np.vectorize(lambda a, b: int(a) | (int(b) << 32), otypes=[object])(words[0], words[1])
    hi = np.vectorize(lambda a, b: (int(a) | (int(b) << 32)) & 0xFFFFFFFFFFFFFFFF, otypes=[object])(
        words[2], words[3])
    out.append(lo.astype(np.uint64))
    out.append(hi.astype(np.uint64))
    return out[0], out[1]


def allreduce_buckets(S1, S2_lo, S2_hi, count, group=None):
    """Sum bucket arrays over all ranks of `group` (torch.distributed); returns new numpy arrays."""
    import torch
    import torch.distributed as dist

    s1 = torch.from_numpy(np.ascontiguousarray(S1, dtype=np.int64).copy())
    cnt = torch.from_numpy(np.ascontiguousarray(count, dtype=np.int64).copy())
    limbs = torch.from_numpy(np.ascontiguousarray(_limbs(np.asarray(S2_lo, np.uint64),
                                                         np.asarray(S2_hi, np.uint64))))
    for t in (s1, cnt, limbs):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    lo, hi = _unlimb(limbs.numpy())
    return s1.numpy(), lo.reshape(np.shape(S2_lo)), hi.reshape(np.shape(S2_hi)), cnt.numpy()


def shard(slots_per_rank: int, rank: int) -> int:
    """Global id of this rank's first slot under weak scaling (fixed slots per rank)."""
    return rank * slots_per_rank
