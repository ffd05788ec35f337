"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas).

Each rank reports its own work and time; the job's throughput is the work of
all ranks over the slowest rank's time, and every rank sees the same value.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    try:
        units = [3.0e9, 5.0e9][rank]
        seconds = [2.0, 4.0][rank]
        value, tmax = bench.job_throughput(dist, torch.device("cpu"), units, seconds)
        dist.barrier()
        q.put((rank, value, tmax))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_work_over_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax in out:
        assert tmax == 4.0
        assert value == pytest.approx(8.0e9 / 4.0, rel=1e-15)


def test_single_process_passes_values_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(None, None, 6.0, 3.0) == (2.0, 3.0)
