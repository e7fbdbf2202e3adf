"""The bench's whole-job figures at N > 1 (world size 2, gloo, CPU): the timed and end-to-end
seconds are the slowest rank's, the site updates and retained replications of a step are summed
over the ranks."""
import json
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


# per rank: timed seconds, site updates of one step, retained replications, end-to-end seconds
RANKS = [(0.9, 39436027500, 14982258, 0.25), (1.2, 39436030000, 14982301, 0.21)]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.reduce_over_ranks(dist, "cpu", *RANKS[rank])
    with open(f"{out}.{rank}", "w") as f:
        json.dump(got, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_the_summed_work(tmp_path):
    out = str(tmp_path / "reduced")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    want = [max(r[0] for r in RANKS), float(sum(r[1] for r in RANKS)),
            float(sum(r[2] for r in RANKS)), max(r[3] for r in RANKS)]
    for rank in range(2):
        with open(f"{out}.{rank}") as f:
            assert json.load(f) == want          # every rank holds the same whole-job figures


def test_one_process_keeps_its_own_figures():
    assert bench.reduce_over_ranks(None, "cpu", *RANKS[1]) == (1.2, 39436030000.0, 14982301.0, 0.21)
