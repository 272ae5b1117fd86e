"""Launch shapes of the smoother and residual kernels: every shape a level
allows gives the oracle's V-cycle within the FP64 bar, and the autotuner's
choices keep the parity bars and are reused from its cache."""

import numpy as np
import pytest

from conftest import oracle_iterate
from oracle import oracle as O
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_params(prm, **kw):
    d = dict(delta=prm.delta, beta=prm.beta, omega=prm.omega, s_min=prm.s_min,
             s_max=prm.s_max, d_max=prm.d_max, coarsen_target=prm.coarsen_target,
             max_levels=prm.max_levels, dense_cap=prm.dense_cap,
             min_rate=prm.min_coarsen_rate)
    d.update(kw)
    return d


CASES = {
    "lognormal_3lev": (lambda: P.lognormal3d((28, 24, 20), seed=1), {"coarsen_target": 300}),
    "laplace2d_64": (lambda: P.laplace2d_random_rhs(64), {"coarsen_target": 200}),
    "hub_graph2d_48": (lambda: P.hub_graph2d(48), {"coarsen_target": 100}),
}


SWEEP = amg.AMG_SHAPE_SWEEP


def _vcycle_err(solver, H, r):
    z = solver.vcycle(torch.from_numpy(np.ascontiguousarray(r)).cuda())
    torch.cuda.synchronize()
    z_or = H.vcycle(r)
    return np.abs(z.cpu().numpy() - z_or).max() / np.abs(z_or).max()


@pytest.mark.parametrize("case", list(CASES))
def test_every_shape_matches_oracle(case):
    maker, over = CASES[case]
    p = maker()
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=p.dim, **over)
    try:
        H = O.Hierarchy(p.row_ptr, p.col, p.val, _oracle_params(solver.params))
        _, levels = solver.info()
        r = np.random.default_rng(7).standard_normal(p.n)
        tried = 0
        for l in range(len(levels) - 1):
            rule = levels[l]["lanes_per_row"]
            for lanes, threads in ((0, 0), (1, 0), (2, 0), (4, 0), (8, 0), (1, 128), (4, 128),
                                   (8, 128), (2 | SWEEP, 0), (8 | SWEEP, 128)):
                try:
                    solver.set_level_shape(l, lanes, threads)
                except amg.AmgError as e:
                    assert (lanes == 0 or lanes & SWEEP) and e.code == amg.AMG_EINVAL
                    continue
                info_l = solver.info()[1][l]
                assert info_l["lanes_per_row"] == lanes & ~SWEEP
                assert info_l["sweep"] == (1 if lanes & SWEEP else 0)
                assert info_l["threads_per_block"] == (threads or 256)
                assert _vcycle_err(solver, H, r) <= 1e-12, (l, lanes, threads)
                tried += 1
            solver.set_level_shape(l, rule)
        assert tried >= 7 * (len(levels) - 1)
        # a mixed assignment through the solve (CUDA graphs rebuilt)
        for l in range(len(levels) - 1):
            solver.set_level_shape(l, (1, 2, 4, 8)[l % 4])
        x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-10, maxit=300)
        assert rc == amg.AMG_OK
        xo, it_o, _, _ = H.pcg(p.b, tol=1e-10, maxit=300)
        assert abs(info["iterations"] - it_o) <= 1
        xo = oracle_iterate(H, p.b, info["iterations"], it_o, xo)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        # the float32 V-cycle under the same shapes
        solver.set_precision(amg.AMG_FP32_IN_FP64)
        x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-8, maxit=300)
        assert rc == amg.AMG_OK and info["true_rel_residual"] <= 1.05e-8
    finally:
        solver.close()


def _own_width_entries(level):
    """Entries of a level in the sliced layout with per-slice widths: rows in
    the smoothing order (colour, then aggregate, then index), 32-row slices,
    each padded to its longest row; and the same with one common width."""
    n = level["n"]
    lens = np.diff(level["row_ptr"]) - 1
    agg = np.where(level["agg"] >= 0, level["agg"], np.iinfo(np.int32).max)
    order = np.lexsort((np.arange(n), agg, level["colour"]))
    ns = (n + 31) // 32
    padded = np.zeros(ns * 32, dtype=np.int64)
    padded[:n] = lens[order]
    kmax = padded.reshape(ns, 32).max(axis=1)
    return int(32 * kmax.sum()), int(32 * ns * lens.max())


def test_per_slice_width_layout_of_varying_levels():
    # Coarse levels whose rows vary in length keep a copy of their entries in
    # 32-row slices padded only to each slice's longest row, for the staged
    # kernels; the fine 7-point level keeps the common width.  The copy's size
    # follows from the oracle's levels, and the staged kernels on it give the
    # oracle's V-cycle, in FP64 to the parity bar and in FP32 through a solve,
    # over colours that start inside a slice and blocks cut short at the end
    # of a level.
    p = P.anisotropic3d((48, 48, 48), seed=0)
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=p.dim)
    try:
        H = O.Hierarchy(p.row_ptr, p.col, p.val, _oracle_params(solver.params))
        _, levels = solver.info()
        assert levels[0]["compact"] == 0
        compact = []
        for l in range(len(levels) - 1):
            own, common = _own_width_entries(H.level(l))
            want = 10 * common > 11 * own
            assert levels[l]["compact"] == int(want), l
            assert levels[l]["staged_entries"] == (own if want else common), l
            if want:
                compact.append(l)
        assert compact and compact[0] == 1
        r = np.random.default_rng(11).standard_normal(p.n)
        staged = 0
        for l in range(len(levels) - 1):
            try:
                solver.set_level_shape(l, 0)
                staged += l in compact
            except amg.AmgError:
                pass
        assert staged >= 1
        assert _vcycle_err(solver, H, r) <= 1e-12
        x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-10, maxit=300)
        assert rc == amg.AMG_OK
        xo, it_o, _, _ = H.pcg(p.b, tol=1e-10, maxit=300)
        assert abs(info["iterations"] - it_o) <= 1
        xo = oracle_iterate(H, p.b, info["iterations"], it_o, xo)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        solver.set_precision(amg.AMG_FP32_IN_FP64)
        x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-8, maxit=300)
        assert rc == amg.AMG_OK and info["true_rel_residual"] <= 1.05e-8
    finally:
        solver.close()


def test_carveout_keeps_the_vcycle_bit_identical():
    # The shared-memory carveout of the staged kernels changes only how the
    # SM splits its L1/shared array: the V-cycle is bit-identical for every
    # value, the level info reports it, and it is refused where it has no
    # meaning.
    maker, over = CASES["lognormal_3lev"]
    p = maker()
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=p.dim, **over)
    try:
        _, levels = solver.info()
        r = torch.from_numpy(np.random.default_rng(5).standard_normal(p.n)).cuda()
        staged = []
        for l in range(len(levels) - 1):
            try:
                solver.set_level_shape(l, 0)
                staged.append(l)
            except amg.AmgError:
                pass
        assert staged
        z0 = solver.vcycle(r).cpu().numpy()
        for pct in (0, 44, 58, 72, 100, -1):
            for l in staged:
                solver.set_level_carveout(l, pct)
                assert solver.info()[1][l]["carveout"] == pct
            z = solver.vcycle(r).cpu().numpy()
            assert np.array_equal(z, z0), pct
        for bad in (-2, 101):
            with pytest.raises(amg.AmgError) as e:
                solver.set_level_carveout(staged[0], bad)
            assert e.value.code == amg.AMG_EINVAL
        solver.set_level_shape(staged[0], 4)
        assert solver.info()[1][staged[0]]["carveout"] == -1
        with pytest.raises(amg.AmgError) as e:
            solver.set_level_carveout(staged[0], 50)
        assert e.value.code == amg.AMG_EINVAL
        with pytest.raises(amg.AmgError) as e:
            solver.set_level_carveout(len(levels) - 1, 50)
        assert e.value.code == amg.AMG_EINVAL
    finally:
        solver.close()


def test_shape_errors():
    p = P.laplace2d_random_rhs(32)
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=2, coarsen_target=100)
    try:
        nlev = solver.info()[0]["num_levels"]
        for l, lanes, threads in ((-1, 4, 0), (nlev - 1, 4, 0), (0, 3, 0), (0, 16, 0), (0, 17, 0),
                                  (0, 4, 64), (0, 0, 128), (0, SWEEP, 0), (0, 3 | SWEEP, 0),
                                  (0, 0x200 | 4, 0)):
            with pytest.raises(amg.AmgError) as e:
                solver.set_level_shape(l, lanes, threads)
            assert e.value.code == amg.AMG_EINVAL
    finally:
        solver.close()


@pytest.mark.parametrize("precision", [amg.AMG_FP64, amg.AMG_FP32_IN_FP64])
def test_autotuned_shapes_keep_parity_and_are_cached(precision):
    p = P.lognormal3d((40, 36, 32), seed=4)
    a = amg.AMG(p.row_ptr, p.col, p.val, dim=3, precision=precision, autotune=1,
                coarsen_target=300)
    try:
        sa, la = a.info()
        shapes = [l["lanes_per_row"] for l in la[:-1]]
        assert all(s in (0, 1, 2, 4, 8) for s in shapes)
        shapes = [(l["lanes_per_row"], l["threads_per_block"], l["sweep"]) for l in la[:-1]]
        H = O.Hierarchy(p.row_ptr, p.col, p.val, _oracle_params(a.params))
        xo, it_o, _, _ = H.pcg(p.b, tol=1e-10, maxit=300)
        if precision == amg.AMG_FP64:
            r = np.random.default_rng(3).standard_normal(p.n)
            assert _vcycle_err(a, H, r) <= 1e-12
            x, rc, info = a.solve(torch.from_numpy(p.b).cuda(), tol=1e-10, maxit=300)
            assert rc == amg.AMG_OK and abs(info["iterations"] - it_o) <= 1
            xo = oracle_iterate(H, p.b, info["iterations"], it_o, xo)
            assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        else:
            x, rc, info = a.solve(torch.from_numpy(p.b).cuda(), tol=1e-8, maxit=300)
            assert rc == amg.AMG_OK and info["true_rel_residual"] <= 1.05e-8
        # a second setup of the same matrix takes every shape from the cache
        b = amg.AMG(p.row_ptr, p.col, p.val, dim=3, precision=precision, autotune=1,
                    coarsen_target=300)
        try:
            sb, lb = b.info()
            assert [(l["lanes_per_row"], l["threads_per_block"], l["sweep"]) for l in lb[:-1]] == shapes
            assert sb["autotune_ms"] == 0.0
        finally:
            b.close()
    finally:
        a.close()


# ---------------------------------------------------------------------------
# smoothing sweeps as one dependency-driven kernel each
# ---------------------------------------------------------------------------

SWEEP_CASES = {
    "lognormal_deep": (lambda: P.lognormal3d((40, 36, 32), seed=4), {"coarsen_target": 60}),
    "layered": (lambda: P.layered3d((24, 24, 28), seed=3), {"coarsen_target": 100}),
    "hub_graph2d_48": (lambda: P.hub_graph2d(48), {"coarsen_target": 100}),
}


@pytest.mark.parametrize("case", list(SWEEP_CASES))
def test_sweep_kernel_gives_the_pass_kernels_values(case):
    # the sweep updates every row exactly as the one-launch-per-pass kernels
    # of the same lanes and block size do: identical V-cycles, on repeated
    # launches (the epochs of the never-reset flags advance), within the
    # oracle bar, and through whole solves in both precisions
    maker, over = SWEEP_CASES[case]
    p = maker()
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=p.dim, **over)
    try:
        H = O.Hierarchy(p.row_ptr, p.col, p.val, _oracle_params(solver.params))
        _, levels = solver.info()
        rng = np.random.default_rng(5)
        r = torch.from_numpy(rng.standard_normal(p.n)).cuda()
        swept = 0
        for l in range(1, len(levels) - 1):
            for lanes, threads in ((2, 0), (4, 128), (8, 0), (1, 128)):
                solver.set_level_shape(l, lanes, threads)
                z_pass = solver.vcycle(r).cpu().numpy()
                try:
                    solver.set_level_shape(l, lanes | SWEEP, threads)
                except amg.AmgError as e:
                    assert e.code == amg.AMG_EINVAL
                    continue
                for _ in range(3):
                    z_sweep = solver.vcycle(r).cpu().numpy()
                    assert np.array_equal(z_sweep, z_pass), (l, lanes, threads)
                swept += 1
            # leave the sweep on for this level
            solver.set_level_shape(l, 4 | SWEEP)
        assert swept >= 1
        z = solver.vcycle(r).cpu().numpy()
        z_or = H.vcycle(r.cpu().numpy())
        assert np.abs(z - z_or).max() <= 1e-12 * np.abs(z_or).max()
        b = torch.from_numpy(p.b).cuda()
        x, rc, info = solver.solve(b, tol=1e-10, maxit=300)
        assert rc == amg.AMG_OK
        xo, it_o, _, _ = H.pcg(p.b, tol=1e-10, maxit=300)
        assert abs(info["iterations"] - it_o) <= 1
        xo = oracle_iterate(H, p.b, info["iterations"], it_o, xo)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        solver.set_precision(amg.AMG_FP32_IN_FP64)
        for l in range(1, len(levels) - 1):
            solver.set_level_shape(l, 4 | SWEEP)
        x, rc, info = solver.solve(b, tol=1e-8, maxit=300)
        assert rc == amg.AMG_OK and info["true_rel_residual"] <= 1.05e-8
    finally:
        solver.close()


def test_sweep_graph_loop_matches_host_loop():
    # the same sweeps launched from the device-side loop graph and from the
    # host-driven loop give identical iterates
    p = P.lognormal3d((36, 30, 28), seed=9)
    out = []
    for device_loop in (1, 0):
        solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, coarsen_target=80,
                         device_loop=device_loop)
        try:
            nlev = solver.info()[0]["num_levels"]
            for l in range(1, nlev - 1):
                solver.set_level_shape(l, 2 | SWEEP, 128)
            x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-10, maxit=300)
            assert rc == amg.AMG_OK and info["device_loop"] == device_loop
            out.append((x.cpu().numpy(), info["iterations"]))
        finally:
            solver.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0].view(np.uint64), out[1][0].view(np.uint64))
