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


def _rank_dies(rank: int, world: int, port: int, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), BENCH_PG_TIMEOUT_S="20")
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    if rank == 1:
        os._exit(3)                 # leaves between steps, with nothing in flight
    try:
        d.barrier()
        d.max(1.0)
        out[rank] = "no error"
    except Exception as e:          # the peer's loss surfaces as an error
        out[rank] = type(e).__name__
    finally:
        try:
            d.close()
        except Exception:
            pass


def test_a_dead_rank_ends_the_others_collectives_with_an_error():
    port = _free_port()
    ctx = multiprocessing.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=120)
        alive = [pr for pr in procs if pr.is_alive()]
        for pr in alive:
            pr.kill()
        assert not alive, "the surviving rank hung"
        assert procs[1].exitcode == 3
        assert 0 in out and out[0] != "no error"

