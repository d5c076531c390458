"""The bench's multi-rank path on CPU: two gloo ranks (world_size 2) agree on the slowest rank's
time and on the whole-job rate.  Replicas do the same work on each rank, so the only exchange
is this one reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 100.0 + 50.0 * rank                 # rank 1 is the slower one
    t = bench.max_over_ranks(t_local, world, "cpu")
    rate = bench.whole_job_rate(30000, world, 5, t)
    out[rank] = (t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == 150.0
        assert rate == pytest.approx(2 * 30000 * 5 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(10, 1, 2, 1000.0) == pytest.approx(20.0)
