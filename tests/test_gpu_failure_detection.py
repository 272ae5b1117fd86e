"""Failure detection without a GPU fault: the staged kernels' bounded wait,
run against an mbarrier that no copy completes, gives up after its poll limit,
records AMG_ETIMEOUT and returns; the device stays usable."""

import numpy as np
import pytest

from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_times_out_and_reports():
    times = {}
    for polls in (1024, 16384):
        status, ms = amg.amg_selftest_bounded_wait(polls)
        assert status == amg.AMG_ETIMEOUT
        times[polls] = ms
    # the time grows with the limit (the wait really polls), and stays short
    assert times[16384] > times[1024]
    assert times[16384] < 5000.0
    per_poll_us = 1e3 * (times[16384] - times[1024]) / (16384 - 1024)
    print(f"\nbounded wait: {per_poll_us:.3f} us per poll; the kernels' limit of 2^18 polls "
          f"gives up after about {per_poll_us * 2**18 / 1e6:.2f} s")


def test_device_is_usable_after_a_timeout():
    status, _ = amg.amg_selftest_bounded_wait(2048)
    assert status == amg.AMG_ETIMEOUT
    p = P.laplace2d_random_rhs(32)
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=2, coarsen_target=100)
    try:
        x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-10)
        assert rc == amg.AMG_OK and info["true_rel_residual"] <= 1.5e-10
    finally:
        solver.close()
