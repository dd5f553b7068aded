"""The multi-rank leg of bench.py on CPU: two gloo ranks, replicas only.

Each rank runs its own replica of the batch; the only exchange is the max of
the per-rank step times after the timed region, and the job rate counts every
rank's queries against the slowest rank.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [10.0 + rank, 3.0 - rank]          # rank 1 is slower on the first timing only
    got = bench.max_over_ranks(mine, dist, None)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == [11.0, 3.0] and out[1] == [11.0, 3.0]


def test_job_rate_is_weak_scaling():
    import bench
    # 4,096 queries per rank, two ranks, slowest step 4 ms -> 2,048,000 queries/s
    assert bench.job_rate(4096, 2, 4.0) == pytest.approx(2.048e6)
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
