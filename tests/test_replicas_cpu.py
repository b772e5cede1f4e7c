"""The multi-GPU path of bench.py is replicas: one process per GPU, each with
its own batch of trajectories, no data exchange, timing combined as the
maximum over ranks.  The host side of that runs here as two gloo processes
on the CPU: both ranks get the maximum, and the ranks' inputs differ."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = (bench.max_over_ranks(1.5 + rank, world, "cpu"),
                     [bench.replica_seed(b, rank) for b in range(8)])
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_maximum_time_and_distinct_inputs():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    seeds = res[0][1] + res[1][1]
    assert len(set(seeds)) == len(seeds)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
