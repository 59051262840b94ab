"""Replica aggregation of the benchmark across ranks (gloo, two CPU
processes): the job time is the slowest rank's, the value counts every
rank's updates."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms_local = [120.0, 200.0][rank]  # rank 1 is the slow one
        ms_max, value = bench.combine_ranks(ms_local, 1_000_000, dist)
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_processes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in got:
        assert ms_max == 200.0
        assert value == pytest.approx(2 * 1_000_000 / 0.2)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench

    ms_max, value = bench.combine_ranks(50.0, 10_000)
    assert ms_max == 50.0 and value == pytest.approx(10_000 / 0.05)
