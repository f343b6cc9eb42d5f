"""The multi-process (replicas) reduction of bench.py on CPU: two gloo ranks, each timing its own replica.

With N GPUs every rank advances an independent replica of the workload; the job's time is the slowest rank's
and its work is the sum over ranks. This checks that reduction with a real two-rank process group.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        t, u = bench.reduce_timing(1.0 + rank, 10 * (rank + 1), world)
        out[rank] = (t, u)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_work():
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {0: (2.0, 30.0), 1: (2.0, 30.0)}


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(1.5, 7, 1) == (1.5, 7)
