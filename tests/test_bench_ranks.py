"""The multi-rank accounting of bench.py (replicas, one process per GPU) on CPU:
two gloo ranks agree on the slowest rank's time, and the whole-job rate counts the
units of every rank over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.0 + rank          # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, dist, "cpu")
        out[rank] = (tmax, bench.job_rate(200, tmax, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    tmax, rate = res[0]
    assert tmax == 2.0
    assert rate == pytest.approx(2 * 200 / 2.0)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(10, 2.0, 1) == 5.0
