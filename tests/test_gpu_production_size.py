"""Element-wise parity with the library's default parameters on grids large
enough to run the production paths: fine-level grids of many waves of blocks,
coarsest levels of thousands of rows (coarsening target 5000, so the blocked
multi-panel Cholesky inverse), the autotuned launch shapes and the device-side
iteration loop.

Bars as in test_gpu_parity: aggregate maps, colours, coarse patterns and
Galerkin values bit-exact on every level; the FP64 V-cycle within 1e-12 of the
oracle's in the max norm; PCG iterations within 1 and solutions within 1e-9 at
a 1e-10 relative residual.
"""

import numpy as np
import pytest

from conftest import oracle_iterate
from oracle import oracle as O
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    # 262,144 rows: 1024 fine-level blocks per pass, 4 levels
    "lognormal_64": lambda: P.lognormal3d((64, 64, 64), seed=0),
    # layers of contrast 1e6: isolated vertices at the interfaces
    "layered_48": lambda: P.layered3d((48, 48, 48), seed=0),
    # z-couplings x 1e-3: planar aggregates, more levels
    "anisotropic_48": lambda: P.anisotropic3d((48, 48, 48), seed=0),
}


@pytest.fixture(scope="module", params=list(CASES))
def big(request):
    p = CASES[request.param]()
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, autotune=1)
    prm = solver.params
    H = O.Hierarchy(p.row_ptr, p.col, p.val,
                    dict(delta=prm.delta, beta=prm.beta, omega=prm.omega, s_min=prm.s_min,
                         s_max=prm.s_max, d_max=prm.d_max, coarsen_target=prm.coarsen_target,
                         max_levels=prm.max_levels, dense_cap=prm.dense_cap,
                         min_rate=prm.min_coarsen_rate))
    yield request.param, p, solver, H
    solver.close()


def test_default_parameters_reach_the_production_paths(big):
    name, p, solver, H = big
    summary, levels = solver.info()
    assert summary["num_levels"] >= 3, name
    # a coarsest level of more than one 32-column panel of the blocked inverse
    assert summary["coarsest_n"] > 64, summary["coarsest_n"]
    # the fine level runs many waves of blocks on 152 SMs
    assert p.n // 256 > 152 * 2


def test_hierarchy_bit_exact_at_default_parameters(big):
    name, p, solver, H = big
    summary, levels = solver.info()
    assert summary["num_levels"] == H.num_levels
    for l in range(H.num_levels):
        g, o = solver.level(l), H.level(l)
        assert g["n"] == o["n"] and g["nnz"] == o["nnz"], (name, l)
        assert np.array_equal(g["row_ptr"], o["row_ptr"])
        assert np.array_equal(g["col"], o["col"])
        assert np.array_equal(g["val"].view(np.uint64), o["val"].view(np.uint64)), (name, l)
        if l < H.num_levels - 1:
            assert np.array_equal(g["agg"], o["agg"]), (name, l)
            assert np.array_equal(g["colour"], o["colour"]), (name, l)


def test_vcycle_matches_oracle_at_default_parameters(big):
    name, p, solver, H = big
    rng = np.random.default_rng(7)
    for r in (p.b, rng.standard_normal(p.n)):
        z_or = H.vcycle(r)
        z = solver.vcycle(torch.from_numpy(np.ascontiguousarray(r)).cuda())
        torch.cuda.synchronize()
        err = np.abs(z.cpu().numpy() - z_or).max()
        assert err <= 1e-12 * np.abs(z_or).max(), (name, err / np.abs(z_or).max())


def test_pcg_matches_oracle_at_default_parameters(big):
    name, p, solver, H = big
    b = torch.from_numpy(p.b).cuda()
    x, rc, info = solver.solve(b, tol=1e-10, maxit=500)
    assert rc == amg.AMG_OK, info
    assert info["device_loop"] in (1, 2)
    xo, it_o, _, _ = H.pcg(p.b, tol=1e-10, maxit=500)
    assert abs(info["iterations"] - it_o) <= 1, (name, info["iterations"], it_o)
    xg = x.cpu().numpy()
    xo = oracle_iterate(H, p.b, info["iterations"], it_o, xo)
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), name
    r = p.b - O.spmv(p.row_ptr, p.col, p.val, xg)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(p.b)


def test_fp32_in_fp64_at_default_parameters(big):
    name, p, solver, H = big
    b = torch.from_numpy(p.b).cuda()
    solver.set_precision(amg.AMG_FP32_IN_FP64)
    try:
        x, rc, info = solver.solve(b, tol=1e-8, maxit=500)
    finally:
        solver.set_precision(amg.AMG_FP64)
    assert rc == amg.AMG_OK
    r = p.b - O.spmv(p.row_ptr, p.col, p.val, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.05e-8 * np.linalg.norm(p.b)


def test_blocked_inverse_at_production_size():
    # one directly solved level of 4352 rows (136 panels of 32 columns, 68
    # tiles of 64): a 3D grid graph with random weights plus a positive shift;
    # the solve applies the blocked inverse and matches numpy's dense solve
    shape = (16, 16, 17)
    n = int(np.prod(shape))
    rng = np.random.default_rng(4)
    rows, cols, vals = [], [], []
    strides = (1, 16, 256)
    w = {}
    for i in range(n):
        co = (i % 16, (i // 16) % 16, i // 256)
        for a in range(3):
            if co[a] + 1 < shape[a]:
                j = i + strides[a]
                w[(i, j)] = w[(j, i)] = 0.5 + rng.random()
    diag = np.full(n, 0.0)
    for (i, j), v in w.items():
        diag[i] += v
    diag += 0.05 + rng.random(n)
    ent = [(i, j, -v) for (i, j), v in w.items()] + [(i, i, diag[i]) for i in range(n)]
    ent.sort()
    rp = np.zeros(n + 1, dtype=np.int32)
    for i, _, _ in ent:
        rp[i + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    ci = np.array([e[1] for e in ent], dtype=np.int32)
    va = np.array([e[2] for e in ent], dtype=np.float64)
    solver = amg.AMG(rp, ci, va, dim=3)   # coarsening target 5000 > n: one level
    try:
        assert solver.info()[0]["num_levels"] == 1
        M = np.zeros((n, n))
        M[np.repeat(np.arange(n), np.diff(rp)), ci] = va
        b = rng.standard_normal(n)
        z = solver.vcycle(torch.from_numpy(b).cuda())
        torch.cuda.synchronize()
        ref = np.linalg.solve(M, b)
        cond = np.linalg.cond(M)
        assert np.abs(z.cpu().numpy() - ref).max() <= 1e-13 * cond * np.abs(ref).max()
    finally:
        solver.close()
