"""bench.py's multi-rank bookkeeping on CPU: two gloo ranks, the step time
that counts is the slowest rank's, and the rate is all ranks' work over it."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        slowest = bench.rank_max(ms, dist)
        rate = bench.whole_job_rate(1e9, world, slowest / 1e3)
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, rate = res[0]
    assert slowest == 15.0
    assert rate == pytest.approx(2 * 1e9 / 0.015)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.5, None) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
