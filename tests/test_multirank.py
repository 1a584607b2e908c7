"""The N > 1 path of the bench (replicas: every rank runs the whole workload
on its own GPU, no data-path collective) on CPU with two gloo ranks: the
timing is the slowest rank's on every rank, and the job's value counts the
work of all ranks over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")  # rank 1 is slower
        out[rank] = (ms, bench.job_value(world, 1e9, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0  # the slowest rank's time everywhere
    assert res[0][1] == pytest.approx(2 * 1e9 / 0.015)  # both ranks' work over that time


def test_single_process_passthrough():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 420 * 2.0 ** 28, 4.37) == pytest.approx(420 * 2.0 ** 28 / 0.00437)
