"""Serving (continuous batching) through the C ABI: amg_server_create,
amg_submit, amg_poll.  Each result must be exactly the one a standalone
setup + solve gives for the same request, whatever else was in flight; the
residual is checked with the oracle's own SpMV."""

import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-8


def _drain(server, tickets, timeout_s=180.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = server.poll(t)
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout_s, "requests did not finish"
        time.sleep(0.002)
    return out


def _standalone(p, server_params):
    prm = server_params.params
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, precision=prm.precision,
                     coarsen_target=prm.coarsen_target, dense_cap=prm.dense_cap,
                     autotune=prm.autotune, aggregation_tile=prm.aggregation_tile)
    x = np.zeros(p.n)
    rc, info = solver.solve_host(p.b, x, tol=TOL, maxit=server_params.maxit)
    solver.close()
    return rc, x, info


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = [P.serving_request(k, lo=8, hi=28) for k in range(10)]
    # the device-side iteration loop here (the server's default is the
    # host-stepped loop, which the next test runs)
    server = amg.Server(dim=3, max_slots=4, setup_threads=3, device_loop=1)
    tickets = [server.submit(p.row_ptr, p.col, p.val, p.b, TOL) for p in reqs]
    res = _drain(server, tickets)
    st = server.stats()
    params = server.params
    server.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 2 <= st["peak_running"] <= 4          # several in flight, never more than the slots
    for p, t in zip(reqs, tickets):
        rc, x, info, times = res[t]
        assert rc == amg.AMG_OK
        assert info["true_rel_residual"] <= 1.5 * TOL
        assert info["device_loop"] == 1      # the iteration loop ran as one device-side graph
        r = p.b - O.spmv(p.row_ptr, p.col, p.val, x)
        assert np.linalg.norm(r) <= 1.05 * TOL * np.linalg.norm(p.b)
        assert times["total_ms"] >= times["solve_ms"] >= 0 and times["hbm_bytes"] > 0
        rc1, x1, info1 = _standalone(p, params)
        assert rc1 == amg.AMG_OK and info1["iterations"] == info["iterations"]
        assert np.array_equal(x, x1), p.name


def test_tuned_shapes_and_tiled_aggregation_in_the_mix():
    # setups tune launch shapes and aggregate in tiles on several threads while
    # other requests solve; shapes of a level signature are shared through the
    # process-wide cache, so a standalone run reproduces each result exactly
    reqs = [P.serving_request(k, lo=12, hi=40) for k in range(60, 84)]
    # (the server's default host-stepped iteration loop: the standalone solves
    # below run the device-side loop, and the two give the same bits)
    server = amg.Server(dim=3, max_slots=8, setup_threads=6, autotune=1, aggregation_tile=512)
    tickets = [server.submit(p.row_ptr, p.col, p.val, p.b, TOL) for p in reqs]
    res = _drain(server, tickets, timeout_s=300.0)
    st = server.stats()
    params = server.params
    server.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for p, t in zip(reqs, tickets):
        rc, x, info, times = res[t]
        assert rc == amg.AMG_OK, amg.amg_last_error()
        assert info["true_rel_residual"] <= 1.5 * TOL
        assert info["device_loop"] == 0
        rc1, x1, info1 = _standalone(p, params)
        assert info1["device_loop"] == 1
        assert rc1 == amg.AMG_OK and info1["iterations"] == info["iterations"]
        assert np.array_equal(x, x1), p.name


def test_admission_by_device_memory():
    # a budget below any request: the server admits one request at a time
    reqs = [P.serving_request(k, lo=8, hi=16) for k in range(20, 25)]
    server = amg.Server(dim=3, max_slots=8, setup_threads=2, hbm_budget_bytes=1.0)
    tickets = [server.submit(p.row_ptr, p.col, p.val, p.b, TOL) for p in reqs]
    res = _drain(server, tickets)
    st = server.stats()
    server.close()
    assert st["peak_running"] == 1 and st["completed"] == len(reqs)
    assert all(res[t][0] == amg.AMG_OK for t in tickets)
    # queued requests waited for the one before them
    assert max(res[t][3]["queue_ms"] for t in tickets[1:]) > 0


def test_failures_are_per_request():
    good = P.serving_request(30, lo=8, hi=14)
    bad = P.serving_request(31, lo=8, hi=14)
    val = bad.val.copy()
    # break the matrix: a negative diagonal fails validation at setup
    val[bad.row_ptr[0]:bad.row_ptr[1]][bad.col[bad.row_ptr[0]:bad.row_ptr[1]] == 0] = -1.0
    server = amg.Server(dim=3, max_slots=2, setup_threads=2)
    tg = server.submit(good.row_ptr, good.col, good.val, good.b, TOL)
    tb = server.submit(bad.row_ptr, bad.col, val, bad.b, TOL)
    res = _drain(server, [tg, tb])
    with pytest.raises(amg.AmgError) as e:
        amg.amg_poll(server.handle, 987654, None)
    assert e.value.code == amg.AMG_ENOTFOUND
    st = server.stats()
    server.close()
    assert res[tg][0] == amg.AMG_OK
    assert res[tb][0] == amg.AMG_EINVAL
    assert st["completed"] == 1 and st["failed"] == 1


def test_destroy_with_work_in_flight():
    reqs = [P.serving_request(k, lo=8, hi=20) for k in range(40, 48)]
    server = amg.Server(dim=3, max_slots=2, setup_threads=1)
    for p in reqs:
        server.submit(p.row_ptr, p.col, p.val, p.b, TOL)
    t0 = time.time()
    server.close()            # running requests finish, queued ones are dropped
    assert time.time() - t0 < 60


@pytest.mark.parametrize("precision", [amg.AMG_FP32_IN_FP64, amg.AMG_FP64])
def test_batched_vcycles_give_each_request_its_own_bits(precision):
    # the scheduler runs the V-cycles of all requests that need one in a tick
    # as shared launches, level by level; every request still gets exactly the
    # bits of its standalone solve, and the same bits as without batching
    reqs = [P.serving_request(k, lo=8, hi=30) for k in range(100, 116)]
    out = {}
    for batch in (1, 0):
        server = amg.Server(dim=3, max_slots=8, setup_threads=4, batch_vcycles=batch,
                            precision=precision)
        tickets = [server.submit(p.row_ptr, p.col, p.val, p.b, TOL) for p in reqs]
        res = _drain(server, tickets)
        st = server.stats()
        params = server.params
        server.close()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        if batch:
            assert st["batched_vcycles"] > 0
            # several requests shared the launches of a batch on average
            assert st["batched_requests"] > st["batched_vcycles"]
        else:
            assert st["batched_vcycles"] == 0
        out[batch] = [res[t] for t in tickets]
    for p, a, b in zip(reqs, out[1], out[0]):
        assert a[0] == b[0] == amg.AMG_OK
        assert a[2]["iterations"] == b[2]["iterations"]
        assert np.array_equal(a[1], b[1]), p.name
        r = p.b - O.spmv(p.row_ptr, p.col, p.val, a[1])
        assert np.linalg.norm(r) <= 1.05 * TOL * np.linalg.norm(p.b)
    for p, a in list(zip(reqs, out[1]))[:4]:
        rc1, x1, info1 = _standalone(p, params)
        assert rc1 == amg.AMG_OK and info1["iterations"] == a[2]["iterations"]
        assert np.array_equal(a[1], x1), p.name
