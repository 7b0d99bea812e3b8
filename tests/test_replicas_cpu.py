"""Replica timing of bench.py under torch.distributed: gloo, world size 2, on CPU.

Every rank solves its own replica; the job time is the maximum over ranks and
the job throughput counts all ranks' elements (weak scaling).
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 1000.0 + 250.0 * rank  # per-rank step time
    job_ms = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (job_ms, bench.job_throughput(world, 100, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo_world2():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        job_ms, thr = out[r]
        assert job_ms == 1250.0
        assert thr == pytest.approx(2 * 100 / 1.25)


def test_single_process_paths():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(1, 32768, 44394.5) == pytest.approx(738.1, rel=1e-3)
