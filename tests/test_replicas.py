"""The multi-process path of bench.py on CPU (gloo, world size 2): replicas
only, a barrier around the timed region and the maximum over ranks."""

import multiprocessing
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    try:
        assert d.world == world and d.rank == rank
        d.barrier()
        m = d.max(float(rank + 1) * 10.0)          # each rank's own timing
        d.barrier()
        # the reference arm prints on rank 0 only; other ranks return at once
        class A:
            steps, warmup, cpu_grid, tol = 1, 0, 8, 1e-8
        if rank != 0:
            assert bench.run_reference(A, d) is None
        out[rank] = m
    finally:
        d.close()


def test_two_rank_max_and_barrier():
    port = _free_port()
    with multiprocessing.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True,
                           start_method="spawn")
        assert dict(out) == {0: 20.0, 1: 20.0}
