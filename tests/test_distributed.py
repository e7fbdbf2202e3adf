"""Slot sharding across ranks (world size 2, gloo, CPU): the exact bucket all-reduce of two slot
halves equals the buckets of one run over all slots (plain, and with a meeting cap and lag 3),
including 128-bit carries of sum G^2."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2608_30239_gb300 import distributed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run(kind, slot_offset=0):
    if kind == "capped_lag3":
        return oracle.coupled_run(3, 20, 90, seed=4, slot_offset=slot_offset, meeting_cap=40, lag=3)
    return oracle.coupled_run(3, 20, 90, seed=4, slot_offset=slot_offset)


def _worker(rank, world, port, P, out, kind):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = synth.tiny_config(2)
    per = P // world
    M = oracle.Model(inst)
    run = _run(kind, distributed.shard(per, rank))
    r = M.run_slots(run, 0, per, 2)
    s1, lo, hi, cnt = distributed.allreduce_buckets(r["S1"], r["S2_lo"], r["S2_hi"], r["count"])
    if rank == 0:
        np.savez(out, S1=s1, lo=lo, hi=hi, cnt=cnt)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["plain", "capped_lag3"])
def test_two_rank_bucket_allreduce(tmp_path, kind):
    P = 1200
    out = str(tmp_path / "r0.npz")
    mp.start_processes(_worker, args=(2, _free_port(), P, out, kind), nprocs=2, start_method="spawn")
    got = np.load(out)
    M = oracle.Model(synth.tiny_config(2))
    ref = M.run_slots(_run(kind), 0, P, 4)
    assert np.array_equal(got["S1"], ref["S1"])
    assert np.array_equal(got["lo"], ref["S2_lo"])
    assert np.array_equal(got["hi"], ref["S2_hi"])
    assert np.array_equal(got["cnt"], ref["count"])


def test_limb_recombination_carries():
    lo = np.array([0xFFFFFFFFFFFFFFFF, 5, 0x8000000000000000], dtype=np.uint64)
    hi = np.array([1, 0, 7], dtype=np.uint64)
    limbs = distributed._limbs(lo, hi) * 3          # three equal ranks
    l2, h2 = distributed._unlimb(limbs)
    for i in range(3):
        total = 3 * ((int(hi[i]) << 64) | int(lo[i]))
        assert int(l2[i]) == total & 0xFFFFFFFFFFFFFFFF
        assert int(h2[i]) == (total >> 64) & 0xFFFFFFFFFFFFFFFF
