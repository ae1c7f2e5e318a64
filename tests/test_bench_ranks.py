"""Multi-rank aggregation of bench.py (one process per GPU, independent replicas), exercised on
the CPU with the gloo backend and two ranks: the job's time is the slowest rank's, its units
are the sum over ranks."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.reduce_over_ranks(100.0 + 50.0 * rank, 202.0 - rank, dist, "cpu")
        out[rank] = (ms, units)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_two_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        assert res[r] == (150.0, 403.0)
