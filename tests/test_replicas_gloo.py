"""The multi-process path of bench.py on CPU: independent replicas, no
data-path collective, whole-job throughput over the slowest rank.  Two gloo
ranks report different local times; both must see the maximum and the sum of
the work of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_local = 100.0 * (rank + 1)            # rank 1 is the slow one
        value, ms_max = bench.replica_throughput(ms_local, 1000, 10, world)
        out[rank] = (value, ms_max)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        value, ms_max = out[r]
        assert ms_max == pytest.approx(200.0)
        assert value == pytest.approx(1000 * 10 * world / 0.2)


def test_single_process_needs_no_group():
    value, ms_max = bench.replica_throughput(50.0, 4, 5, 1)
    assert ms_max == 50.0 and value == pytest.approx(4 * 5 / 0.05)
