"""CPU tests of libamg: the C ABI loads and exports what include/amg.h
declares, input validation, and bit-exact parity of the library's host setup
(strength of connection, Algorithms 1-3, colouring) with the oracle."""

import ctypes
import json
import os
import re

import numpy as np
import pytest

from conftest import graph_from_spec, ROOT
from oracle import oracle as O
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "amg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = amg.lib(build_if_missing=True)
    names = _declared_functions()
    assert "amg_setup" in names and "amg_pcg_solve" in names
    for name in names:
        assert hasattr(L, name), name
        assert name in amg._SIGNATURES, f"binding lacks {name}"


def test_checked_build_exports_the_same_symbols():
    # the checked build (device-side index checks) has the same interface;
    # read with nm so that one process does not load both libraries
    import shutil
    import subprocess
    from paper_1209_0960_gb300 import build as B
    if shutil.which("nm") is None:
        pytest.skip("no nm")
    path = B.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared_functions():
        assert name in syms, name
    assert amg.lib().amg_device_checks() in (0, 1)


def test_debug_column_hook_refused_outside_the_checked_build():
    if amg.lib().amg_device_checks():
        pytest.skip("the loaded library is the checked build")
    assert amg.lib().amg_debug_set_column(None, 1, 0, 0, 10) == amg.AMG_EINVAL
    assert "checked build" in amg.amg_last_error()


def test_params_default_and_errors():
    p = amg.amg_params_default(3)
    assert (p.s_min, p.s_max, p.d_max) == (8, 12, 3)
    assert p.delta == pytest.approx(1 / 3) and p.omega == 1.6
    assert p.device_loop == 1 and p.coarsest_fp32 == 0 and p.autotune == 0
    assert p.launch_overlap == 1 and p.flexible_cg == -1
    assert amg.amg_server_params_default(3).params.device_loop == 0
    p2 = amg.amg_params_default(2)
    assert (p2.s_min, p2.s_max, p2.d_max) == (4, 6, 2)
    with pytest.raises(amg.AmgError) as e:
        amg.amg_params_default(4)
    assert e.value.code == amg.AMG_EINVAL


@pytest.mark.parametrize("bad", ["unsorted", "missing_diag", "nonpositive_diag", "asym", "range"])
def test_aggregate_rejects_malformed_csr(bad):
    p = P.laplace2d_random_rhs(4)
    rp, ci, va = p.row_ptr.copy(), p.col.copy(), p.val.copy()
    if bad == "unsorted":
        ci[rp[5]], ci[rp[5] + 1] = ci[rp[5] + 1], ci[rp[5]]
    elif bad == "missing_diag":
        k = [k for k in range(rp[3], rp[4]) if ci[k] == 3][0]
        ci[k] = ci[k] + 0  # keep, then drop the entry below
        keep = np.ones(len(ci), bool)
        keep[k] = False
        rp = rp.copy()
        rp[4:] -= 1
        ci, va = ci[keep], va[keep]
    elif bad == "nonpositive_diag":
        k = [k for k in range(rp[3], rp[4]) if ci[k] == 3][0]
        va[k] = -1.0
    elif bad == "asym":
        # replace the (0, 1) entry by (0, 2): pattern loses symmetry
        ci = ci.copy()
        k = [k for k in range(rp[0], rp[1]) if ci[k] == 1][0]
        ci[k] = 2
    elif bad == "range":
        ci[-1] = 10_000
    with pytest.raises(amg.AmgError) as e:
        amg.amg_aggregate(rp, ci, va, amg.amg_params_default(2))
    assert e.value.code == amg.AMG_EINVAL
    assert amg.amg_last_error() != ""


with open(os.path.join(os.path.dirname(__file__), "golden", "aggregation_hand.json")) as f:
    _HAND = json.load(f)["cases"]


@pytest.mark.parametrize("case", _HAND, ids=[c["name"] for c in _HAND])
def test_library_aggregation_hand_derived(case):
    rp, ci, va = graph_from_spec(case["graph"])
    prm = amg.amg_params_default(2)
    for k, v in case["params"].items():
        setattr(prm, k, v)
    agg, nc = amg.amg_aggregate(rp, ci, va, prm)
    assert nc == case["nc"] and agg.tolist() == case["agg"]


def _oracle_params(prm):
    return dict(delta=prm.delta, beta=prm.beta, omega=prm.omega, s_min=prm.s_min,
                s_max=prm.s_max, d_max=prm.d_max, coarsen_target=prm.coarsen_target,
                max_levels=prm.max_levels, dense_cap=prm.dense_cap,
                min_rate=prm.min_coarsen_rate)


@pytest.mark.parametrize("maker", [
    lambda: P.laplace2d_random_rhs(64),
    lambda: P.lognormal3d((24, 20, 17), seed=11),
    lambda: P.lognormal3d((16, 16, 16), variance=6.0, corr_len=0.02, seed=3),
    lambda: P.layered3d((18, 18, 22), seed=4),
    lambda: P.anisotropic3d((14, 15, 16), seed=2),
    lambda: P.serving_request(7) if False else P.lognormal3d((19, 23, 17), variance=1.0, corr_len=0.1, seed=7),
], ids=["laplace2d", "lognormal", "lognormal_rough", "layered", "anisotropic", "box"])
def test_library_host_setup_matches_oracle_bit_exactly(maker):
    p = maker()
    prm = amg.amg_params_default(p.dim)
    agg1, n1 = amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    agg2, n2 = O.aggregate(p.row_ptr, p.col, p.val, _oracle_params(prm))
    assert n1 == n2
    assert np.array_equal(agg1, agg2)
    c1, k1 = amg.amg_colour(p.row_ptr, p.col, p.val)
    c2, k2 = O.colour(p.row_ptr, p.col)
    assert k1 == k2 and np.array_equal(c1, c2)


def test_library_host_setup_matches_oracle_on_coarse_levels():
    # the oracle's coarse matrices exercise denser rows, isolated vertices and
    # irregular graphs
    p = P.layered3d((20, 20, 20), seed=9)
    prm = amg.amg_params_default(3)
    H = O.Hierarchy(p.row_ptr, p.col, p.val, dict(_oracle_params(prm), coarsen_target=20))
    assert H.num_levels >= 3
    for l in range(H.num_levels - 1):
        L = H.level(l)
        agg, nc = amg.amg_aggregate(L["row_ptr"], L["col"], L["val"], prm)
        assert nc == L["nc"] and np.array_equal(agg, L["agg"]), l
        col, k = amg.amg_colour(L["row_ptr"], L["col"], L["val"])
        assert k == L["ncolours"] and np.array_equal(col, L["colour"])


@pytest.mark.parametrize("seed", range(4))
def test_library_aggregation_matches_oracle_with_isolated_vertices(seed):
    # strong random contrast: beta raised so that many vertices are isolated
    rng = np.random.default_rng(seed)
    K = np.exp(rng.normal(0.0, 4.0, size=(12, 11, 10)))
    rp, ci, va, b = P.assemble_fv(K, bc=[(1.0, 0.0), (None, None), (None, None)])
    prm = amg.amg_params_default(3)
    prm.beta = 0.02
    _, iso, _, _ = O.strength(rp, ci, va, _oracle_params(prm))
    assert iso.sum() > 20
    agg1, n1 = amg.amg_aggregate(rp, ci, va, prm)
    agg2, n2 = O.aggregate(rp, ci, va, _oracle_params(prm))
    assert n1 == n2 and np.array_equal(agg1, agg2)


_TILED = {
    "lognormal_tile64": (lambda: P.lognormal3d((14, 13, 12), seed=6), 64),
    "lognormal_tile_ragged": (lambda: P.lognormal3d((14, 13, 12), seed=6), 331),
    "layered_tile_plane": (lambda: P.layered3d((16, 16, 10), seed=1), 256),
    "laplace2d_tile1": (lambda: P.laplace2d_random_rhs(12), 1),
    "laplace2d_tile_gt_n": (lambda: P.laplace2d_random_rhs(20), 1000),
    "hub_graph": (lambda: P.hub_graph2d(40), 97),
}


@pytest.mark.parametrize("case", list(_TILED))
def test_library_tiled_aggregation_matches_oracle(case):
    maker, tile = _TILED[case]
    p = maker()
    prm = amg.amg_params_default(p.dim)
    prm.aggregation_tile = tile
    agg1, n1 = amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    agg2, n2 = O.aggregate(p.row_ptr, p.col, p.val, dict(_oracle_params(prm), agg_tile=tile))
    assert n1 == n2 and np.array_equal(agg1, agg2)


@pytest.mark.parametrize("seed", range(2))
def test_library_tiled_aggregation_with_isolated_vertices(seed):
    rng = np.random.default_rng(10 + seed)
    K = np.exp(rng.normal(0.0, 4.0, size=(12, 11, 10)))
    rp, ci, va, b = P.assemble_fv(K, bc=[(1.0, 0.0), (None, None), (None, None)])
    prm = amg.amg_params_default(3)
    prm.beta = 0.02
    prm.aggregation_tile = 150
    agg1, n1 = amg.amg_aggregate(rp, ci, va, prm)
    agg2, n2 = O.aggregate(rp, ci, va, dict(_oracle_params(prm), agg_tile=150))
    assert n1 == n2 and np.array_equal(agg1, agg2)


def test_tiled_aggregation_parameters_are_checked():
    p = P.laplace2d_random_rhs(8)
    prm = amg.amg_params_default(2)
    prm.aggregation_tile = -1
    with pytest.raises(amg.AmgError) as e:
        amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    assert e.value.code == amg.AMG_EINVAL
    prm.aggregation_tile = 16
    prm.aggregation_device = 2
    with pytest.raises(amg.AmgError) as e:
        amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    assert e.value.code == amg.AMG_EINVAL
    prm.aggregation_device = 0
    prm.coarsest_fp32 = 2
    with pytest.raises(amg.AmgError) as e:
        amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    assert e.value.code == amg.AMG_EINVAL
    assert "coarsest_fp32" in amg.amg_last_error()
    prm.coarsest_fp32 = 0
    prm.device_loop = 2
    with pytest.raises(amg.AmgError) as e:
        amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    assert e.value.code == amg.AMG_EINVAL
    assert "device_loop" in amg.amg_last_error()


def test_value_symmetry_is_checked_under_amg_check(monkeypatch):
    p = P.lognormal3d((6, 5, 4), seed=1)
    va = p.val.copy()
    # perturb one off-diagonal entry (0, j) but not (j, 0)
    k = [k for k in range(p.row_ptr[0], p.row_ptr[1]) if p.col[k] != 0][0]
    va[k] *= 1.0 + 1e-12
    prm = amg.amg_params_default(3)
    monkeypatch.delenv("AMG_CHECK", raising=False)
    amg.amg_aggregate(p.row_ptr, p.col, va, prm)          # pattern only: accepted
    monkeypatch.setenv("AMG_CHECK", "1")
    amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)       # symmetric values: accepted
    with pytest.raises(amg.AmgError) as e:
        amg.amg_aggregate(p.row_ptr, p.col, va, prm)
    assert e.value.code == amg.AMG_EINVAL
    assert "not symmetric" in amg.amg_last_error()


def test_tiled_aggregation_does_not_depend_on_host_threads():
    p = P.lognormal3d((16, 15, 14), seed=3)
    prm = amg.amg_params_default(3)
    prm.aggregation_tile = 300
    maps = []
    for t in (1, 3, 0):
        prm.host_threads = t
        maps.append(amg.amg_aggregate(p.row_ptr, p.col, p.val, prm))
    assert all(m[1] == maps[0][1] and np.array_equal(m[0], maps[0][0]) for m in maps)
    prm.host_threads = -1
    with pytest.raises(amg.AmgError):
        amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)


def test_bounded_wait_selftest_rejects_bad_arguments():
    with pytest.raises(amg.AmgError) as e:
        amg.amg_selftest_bounded_wait(-1)
    assert e.value.code == amg.AMG_EINVAL


@pytest.mark.parametrize("name", ["amg_pcg_solve", "amg_pcg_solve_host",
                                  "amg_pcg_solve_host_zero_guess", "amg_bicgstab_solve"])
def test_solve_entry_points_reject_a_null_context(name):
    # argument checks come before any device work, so they run without a GPU
    L = amg.lib()
    b = np.zeros(4)
    x = np.zeros(4)
    info = amg.amg_solve_info()
    rc = getattr(L, name)(None, b.ctypes.data, x.ctypes.data, 1e-8, 10, ctypes.byref(info))
    assert rc == amg.AMG_EINVAL
    assert "null" in amg.amg_last_error()


def test_library_aggregation_of_a_long_chain_has_the_closed_form():
    # the chain of the oracle pin (agg[i] = i // 3, the last single vertex
    # joining the previous aggregate), through the library's host aggregation
    n = 100000
    rows = [[j for j in (i - 1, i, i + 1) if 0 <= j < n] for i in range(n)]
    ci = np.concatenate([np.array(r, np.int32) for r in rows])
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    va = np.where(ci == np.repeat(np.arange(n), np.diff(rp)), 2.0, -1.0)
    agg, nc = amg.amg_aggregate(rp, ci, va, amg.amg_params_default(2))
    expect = np.arange(n) // 3
    expect[-1] = expect[-2]
    assert nc == expect[-1] + 1 and np.array_equal(agg, expect)


@pytest.mark.parametrize("m", [50001, 50002])
def test_library_aggregation_of_a_long_ladder_has_the_closed_form(m):
    # the 2 x m ladder of the oracle pin, through the library's host aggregation
    from test_oracle_pins import _ladder, ladder_closed_form
    rp, ci, va = _ladder(m)
    agg, nc = amg.amg_aggregate(rp, ci, va, amg.amg_params_default(2))
    expect = ladder_closed_form(m)
    assert nc == expect.max() + 1 and np.array_equal(agg, expect)


def test_large_matrix_validation_reports_the_lowest_failing_row():
    # Matrices of 2^20 rows or more are validated on several host threads; the
    # message still names the lowest failing row, whichever chunk holds it.
    n = (1 << 20) + 12345
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0), np.full(n - 1, -1.0)])
    order = np.lexsort((cols, rows))
    rp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    ci, va = cols[order].astype(np.int32), vals[order].copy()
    prm = amg.amg_params_default(1)

    def diag_pos(r):
        return [k for k in range(rp[r], rp[r + 1]) if ci[k] == r][0]

    # errors of the first pass in several chunks: the lowest row wins
    va2 = va.copy()
    for r in (n - 7, 700_001, 300_017):
        va2[diag_pos(r)] = -1.0
    with pytest.raises(amg.AmgError):
        amg.amg_aggregate(rp, ci, va2, prm)
    assert amg.amg_last_error().endswith("non-positive diagonal in row 300017")
    # a pattern error is reported only when every row passes the first pass
    ci3 = ci.copy()
    k = [k for k in range(rp[900_000], rp[900_001]) if ci3[k] == 900_001][0]
    ci3[k] = 900_002   # (900000, 900002) without (900002, 900000)
    with pytest.raises(amg.AmgError):
        amg.amg_aggregate(rp, ci3, va, prm)
    assert "pattern not symmetric at (900000,900002)" in amg.amg_last_error()
    # and the well-formed matrix aggregates: a chain in blocks of s_min = 2
    agg, nc = amg.amg_aggregate(rp, ci, va, prm)
    assert nc > 0 and agg.min() >= 0
