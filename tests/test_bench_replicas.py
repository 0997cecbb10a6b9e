"""Multi-process (replicas only) host logic of bench.py on CPU: two gloo ranks time
different amounts and both report the maximum and the whole-job rate."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_max, rate = bench.replica_rate(100.0 * (rank + 1), steps=3, world=world, device="cpu")
    out[rank] = (ms_max, rate)
    dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ms_max, rate = out[r]
        assert ms_max == pytest.approx(200.0)
        assert rate == pytest.approx(world * 3 / 0.2)


def test_replica_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(250.0, steps=5, world=1) == (250.0, pytest.approx(20.0))
