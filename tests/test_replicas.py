"""The multi-GPU path is replicas only: each rank processes its own stream and the
bench reports all ranks' samples over the slowest rank's time.  The reduction runs
here with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, value = bench.replica_throughput(10.0 * (rank + 1), 1_000_000, dist, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 20.0                                  # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 1_000_000 / 0.020)


def test_replica_throughput_single_process():
    import bench
    ms, value = bench.replica_throughput(5.0, 1000)
    assert ms == 5.0 and value == pytest.approx(1000 / 0.005)
