"""The PCG iteration loop run on the device (one CUDA graph with a WHILE node
whose condition a kernel sets after each update) against the host-driven
loop: the same launches in the same order, so the iterates agree bit for bit,
at convergence and at maxit; and the zero-initial-guess host entry point
against the host entry point with x_0 zeroed."""

import numpy as np
import pytest

from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def problem():
    return P.lognormal3d((30, 26, 22), seed=7)


def _solve(p, device_loop, precision, flexible, tol, maxit):
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, device_loop=device_loop,
                     precision=precision, flexible_cg=flexible)
    try:
        b = torch.from_numpy(p.b).cuda()
        out = []
        for _ in range(2):   # the second solve replays the cached graph
            x, rc, info = solver.solve(b, tol=tol, maxit=maxit)
            torch.cuda.synchronize()
            out.append((x.cpu().numpy(), rc, info))
        return out
    finally:
        solver.close()


@pytest.mark.parametrize("precision,flexible", [(amg.AMG_FP64, 0), (amg.AMG_FP64, 1),
                                                (amg.AMG_FP32_IN_FP64, 0)])
def test_device_loop_matches_host_loop(problem, precision, flexible):
    dev = _solve(problem, 1, precision, flexible, 1e-9, 300)
    host = _solve(problem, 0, precision, flexible, 1e-9, 300)
    for (xd, rcd, infod), (xh, rch, infoh) in zip(dev, host):
        assert rcd == rch == amg.AMG_OK
        assert infod["device_loop"] == 1 and infoh["device_loop"] == 0
        assert infod["iterations"] == infoh["iterations"]
        assert infod["rel_residual"] == infoh["rel_residual"]
        assert np.array_equal(xd.view(np.uint64), xh.view(np.uint64))
    assert np.array_equal(dev[0][0].view(np.uint64), dev[1][0].view(np.uint64))


def test_device_loop_stops_at_maxit(problem):
    dev = _solve(problem, 1, amg.AMG_FP64, 0, 1e-30, 5)
    host = _solve(problem, 0, amg.AMG_FP64, 0, 1e-30, 5)
    for (xd, rcd, infod), (xh, rch, infoh) in zip(dev, host):
        assert rcd == rch == amg.AMG_ENOTCONV
        assert infod["iterations"] == infoh["iterations"] == 5
        assert infod["device_loop"] == 1
        assert np.array_equal(xd.view(np.uint64), xh.view(np.uint64))


def test_device_loop_single_iteration_and_zero_rhs(problem):
    solver = amg.AMG(problem.row_ptr, problem.col, problem.val, dim=3)
    try:
        b = torch.from_numpy(problem.b).cuda()
        x, rc, info = solver.solve(b, tol=1e-30, maxit=1)
        assert rc == amg.AMG_ENOTCONV and info["iterations"] == 1
        x, rc, info = solver.solve(torch.zeros_like(b), tol=1e-8)
        assert rc == amg.AMG_OK and info["iterations"] == 0 and info["device_loop"] == 0
        assert torch.count_nonzero(x).item() == 0
        x, rc, info = solver.solve(b, tol=1e-8)
        assert rc == amg.AMG_OK and info["device_loop"] == 1
        assert info["true_rel_residual"] <= 1.05e-8
    finally:
        solver.close()


def test_zero_guess_host_solve_matches_zeroed_x0(problem):
    solver = amg.AMG(problem.row_ptr, problem.col, problem.val, dim=3)
    try:
        bh = torch.from_numpy(problem.b).pin_memory().numpy()
        x1 = torch.zeros(problem.n, dtype=torch.float64).pin_memory().numpy()
        x2 = torch.full((problem.n,), np.nan, dtype=torch.float64).pin_memory().numpy()
        rc1, i1 = solver.solve_host(bh, x1, tol=1e-10)
        rc2, i2 = solver.solve_host(bh, x2, tol=1e-10, zero_guess=True)
        assert rc1 == rc2 == amg.AMG_OK and i1["iterations"] == i2["iterations"]
        assert np.array_equal(x1.view(np.uint64), x2.view(np.uint64))
    finally:
        solver.close()


def _solve_bi(p, device_loop, precision, tol, maxit):
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, device_loop=device_loop, precision=precision)
    try:
        b = torch.from_numpy(p.b).cuda()
        out = []
        for _ in range(2):   # the second solve replays the cached graph
            x, rc, info = solver.solve_bicgstab(b, tol=tol, maxit=maxit)
            torch.cuda.synchronize()
            out.append((x.cpu().numpy(), rc, info))
        return out
    finally:
        solver.close()


@pytest.mark.parametrize("precision", [amg.AMG_FP64, amg.AMG_FP32_IN_FP64])
@pytest.mark.parametrize("tol,maxit,rc_want", [(1e-9, 300, amg.AMG_OK), (1e-30, 4, amg.AMG_ENOTCONV)])
def test_bicgstab_device_loop_matches_host_loop(problem, precision, tol, maxit, rc_want):
    # BiCGSTAB keeps its scalars on the device: the graph loop and the
    # host-driven loop launch the same kernels and stop at the same point
    dev = _solve_bi(problem, 1, precision, tol, maxit)
    host = _solve_bi(problem, 0, precision, tol, maxit)
    for (xd, rcd, infod), (xh, rch, infoh) in zip(dev, host):
        assert rcd == rch == rc_want
        assert infod["device_loop"] == 1 and infoh["device_loop"] == 0
        assert infod["iterations"] == infoh["iterations"]
        if rc_want == amg.AMG_ENOTCONV:
            assert infod["iterations"] == maxit
        assert infod["rel_residual"] == infoh["rel_residual"]
        assert np.array_equal(xd.view(np.uint64), xh.view(np.uint64))
    assert np.array_equal(dev[0][0].view(np.uint64), dev[1][0].view(np.uint64))


def test_bicgstab_zero_rhs_and_half_step_exit(problem):
    solver = amg.AMG(problem.row_ptr, problem.col, problem.val, dim=3)
    try:
        b = torch.from_numpy(problem.b).cuda()
        x, rc, info = solver.solve_bicgstab(torch.zeros_like(b), tol=1e-8)
        assert rc == amg.AMG_OK and info["iterations"] == 0
        assert torch.count_nonzero(x).item() == 0
        # a loose tolerance that the first half step already meets: one
        # iteration, x = alpha y, and the reported residual is the half step's
        x, rc, info = solver.solve_bicgstab(b, tol=0.9)
        assert rc == amg.AMG_OK and info["iterations"] == 1
        assert info["true_rel_residual"] <= 0.9
    finally:
        solver.close()
