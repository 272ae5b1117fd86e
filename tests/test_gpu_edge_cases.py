"""Degenerate inputs of the method through the C ABI: a single row, rows
without off-diagonals (no aggregate can form), a right-hand side of zero,
disconnected components, decoupled rows inside a grid and a ragged tiny grid
coarsened to many levels -- each against the oracle or a closed form."""

import numpy as np
import pytest
import scipy.sparse as sp

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


def _csr(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64)


def _check_against_oracle(rp, ci, va, b, dim, **over):
    solver = amg.AMG(rp, ci, va, dim=dim, **over)
    try:
        H = O.Hierarchy(rp, ci, va, _oracle_params(solver.params))
        s, levels = solver.info()
        assert s["num_levels"] == H.num_levels
        for l in range(H.num_levels):
            g, o = solver.level(l), H.level(l)
            assert np.array_equal(g["row_ptr"], o["row_ptr"]) and np.array_equal(g["col"], o["col"])
            assert np.array_equal(g["val"].view(np.uint64), o["val"].view(np.uint64))
            if l < H.num_levels - 1:
                assert np.array_equal(g["agg"], o["agg"])
                assert np.array_equal(g["colour"], o["colour"])
        z = solver.vcycle(torch.from_numpy(b).cuda())
        torch.cuda.synchronize()
        z_or = H.vcycle(b)
        assert np.abs(z.cpu().numpy() - z_or).max() <= 1e-12 * np.abs(z_or).max()
        x, rc, info = solver.solve(torch.from_numpy(b).cuda(), tol=1e-10, maxit=300)
        assert rc == amg.AMG_OK
        xo, it_o, _, _ = H.pcg(b, tol=1e-10, maxit=300)
        assert abs(info["iterations"] - it_o) <= 1
        xo = oracle_iterate(H, b, info["iterations"], it_o, xo)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        return s, levels
    finally:
        solver.close()


def test_single_row():
    rp = np.array([0, 1], np.int32)
    ci = np.array([0], np.int32)
    va = np.array([4.0])
    solver = amg.AMG(rp, ci, va, dim=3)
    try:
        assert solver.info()[0]["num_levels"] == 1
        x, rc, info = solver.solve(torch.tensor([2.0], dtype=torch.float64, device="cuda"), tol=1e-12)
        assert rc == amg.AMG_OK and info["iterations"] == 1
        assert x.item() == 0.5
    finally:
        solver.close()


@pytest.mark.parametrize("precision", [amg.AMG_FP64, amg.AMG_FP32_IN_FP64])
def test_diagonal_matrix_forms_no_aggregate(precision):
    # every row lacks an off-diagonal: no aggregate forms, so the hierarchy is
    # one level solved directly
    n = 1000
    d = 1.0 + np.arange(n) / n
    rp, ci, va = _csr(sp.diags(d))
    assert amg.amg_aggregate(rp, ci, va, amg.amg_params_default(3))[1] == 0
    solver = amg.AMG(rp, ci, va, dim=3, coarsen_target=10, precision=precision)
    try:
        assert solver.info()[0]["num_levels"] == 1
        b = np.random.default_rng(0).standard_normal(n)
        x, rc, info = solver.solve(torch.from_numpy(b).cuda(), tol=1e-10)
        assert rc == amg.AMG_OK
        if precision == amg.AMG_FP64:
            # the preconditioner is A^-1 itself
            assert info["iterations"] == 1
            assert np.abs(x.cpu().numpy() - b / d).max() <= 1e-12 * np.abs(b / d).max()
        else:
            # A^-1 applied in float32: a few iterations
            assert info["iterations"] <= 4 and info["true_rel_residual"] <= 1.5e-10
    finally:
        solver.close()


def test_uncoarsenable_level_above_the_dense_cap_is_an_error():
    n = 9000
    rp, ci, va = _csr(sp.diags(np.full(n, 2.0)))
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(rp, ci, va, dim=3, coarsen_target=10)
    assert e.value.code == amg.AMG_EINVAL
    assert "dense_cap" in amg.amg_last_error()


def test_zero_right_hand_side():
    p = P.lognormal3d((12, 11, 10), seed=2)
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, coarsen_target=100)
    try:
        b = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        x, rc, info = solver.solve(b, tol=1e-8)
        assert rc == amg.AMG_OK and info["iterations"] == 0
        assert torch.count_nonzero(x).item() == 0
    finally:
        solver.close()


def test_disconnected_components():
    a = P.laplace2d_random_rhs(24, seed=1)
    c = P.lognormal3d((10, 9, 8), seed=4)
    A = sp.block_diag([sp.csr_matrix((a.val, a.col, a.row_ptr)),
                       sp.csr_matrix((c.val, c.col, c.row_ptr))])
    rp, ci, va = _csr(A)
    b = np.concatenate([a.b, c.b])
    s, levels = _check_against_oracle(rp, ci, va, b, 3, coarsen_target=60)
    assert s["num_levels"] >= 3


def test_decoupled_rows_inside_a_grid():
    # rows whose couplings are removed on both sides (identity-like rows): they
    # are left out of every aggregate and the smoother solves them exactly
    p = P.lognormal3d((14, 12, 10), seed=5)
    A = sp.csr_matrix((p.val, p.col, p.row_ptr)).tolil()
    rng = np.random.default_rng(6)
    cut = rng.choice(p.n, size=40, replace=False)
    for i in cut:
        for j in list(A.rows[i]):
            if j != i:
                A[i, j] = 0.0
                A[j, i] = 0.0
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    rp, ci, va = _csr(A)
    agg, nc = amg.amg_aggregate(rp, ci, va, amg.amg_params_default(3))
    assert (agg[cut] == -1).all()
    _check_against_oracle(rp, ci, va, p.b, 3, coarsen_target=80)


def test_ragged_tiny_grid_many_levels():
    # 3 x 11 cells (33 rows, not a multiple of a 32-row slice) coarsened down
    # to a single row
    K = np.ones((3, 11))
    rp, ci, va, b = P.assemble_fv(K, bc=[(1.0, 0.0), (None, None)])
    s, levels = _check_against_oracle(rp, ci, va, b, 2, coarsen_target=2, min_coarsen_rate=1.0)
    assert s["num_levels"] >= 3


def test_device_resident_matrix_gives_the_same_hierarchy():
    p = P.lognormal3d((16, 15, 14), seed=8)
    host = amg.AMG(p.row_ptr, p.col, p.val, dim=3, coarsen_target=100)
    dev = amg.AMG(torch.from_numpy(p.row_ptr).cuda(), torch.from_numpy(p.col).cuda(),
                  torch.from_numpy(p.val).cuda(), dim=3, coarsen_target=100)
    try:
        sh, _ = host.info()
        sd, _ = dev.info()
        assert sh["num_levels"] == sd["num_levels"]
        for l in range(sh["num_levels"]):
            a, b = host.level(l), dev.level(l)
            assert np.array_equal(a["row_ptr"], b["row_ptr"]) and np.array_equal(a["col"], b["col"])
            assert np.array_equal(a["val"].view(np.uint64), b["val"].view(np.uint64))
        bt = torch.from_numpy(p.b).cuda()
        x1, rc1, i1 = host.solve(bt, tol=1e-10)
        x2, rc2, i2 = dev.solve(bt, tol=1e-10)
        assert rc1 == rc2 == amg.AMG_OK and i1["iterations"] == i2["iterations"]
        assert torch.equal(x1, x2)
    finally:
        host.close()
        dev.close()


def test_indefinite_coarsest_level_is_reported():
    # symmetric with a positive diagonal but indefinite (eigenvalues 3 and -1):
    # the coarsest Cholesky meets a non-positive pivot
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    va = np.array([1.0, 2.0, 2.0, 1.0])
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(rp, ci, va, dim=2)
    assert e.value.code == amg.AMG_ENOTSPD
    # the device keeps working
    p = P.laplace2d_random_rhs(16)
    s = amg.AMG(p.row_ptr, p.col, p.val, dim=2)
    try:
        x, rc, info = s.solve(torch.from_numpy(p.b).cuda(), tol=1e-10)
        assert rc == amg.AMG_OK
    finally:
        s.close()


@pytest.mark.parametrize("n", [31, 33, 64, 97, 130])
def test_coarsest_inverse_against_numpy(n):
    # one directly solved level of n rows: the solve applies the blocked
    # inverse; its result matches a dense solve (tile edges of 32 and 64)
    rng = np.random.default_rng(n)
    B = sp.random(n, n, density=0.2, random_state=int(n)).toarray()
    M = -(np.abs(B) + np.abs(B.T))
    np.fill_diagonal(M, 0.0)
    M += np.diag(-M.sum(axis=1) + 1.0 + rng.random(n))
    rp, ci, va = _csr(M)
    solver = amg.AMG(rp, ci, va, dim=3, coarsen_target=1000)
    try:
        assert solver.info()[0]["num_levels"] == 1
        b = rng.standard_normal(n)
        z = solver.vcycle(torch.from_numpy(b).cuda())
        torch.cuda.synchronize()
        ref = np.linalg.solve(M, b)
        assert np.abs(z.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max() * np.linalg.cond(M)
    finally:
        solver.close()


def test_float32_coarsest_inverse_single_level():
    # one directly solved level, float32 V-cycle: with coarsest_fp32 the
    # inverse is applied as a float32 matrix; the result is A^-1 r up to
    # float32 rounding of the scaled inverse, the right-hand side and the sums
    n = 130
    rng = np.random.default_rng(11)
    B = sp.random(n, n, density=0.2, random_state=11).toarray()
    M = -(np.abs(B) + np.abs(B.T))
    np.fill_diagonal(M, 0.0)
    M += np.diag(-M.sum(axis=1) + 1.0 + rng.random(n))
    rp, ci, va = _csr(M)
    b = rng.standard_normal(n)
    ref = np.linalg.solve(M, b)
    errs = []
    for flag in (0, 1):
        solver = amg.AMG(rp, ci, va, dim=3, coarsen_target=1000, coarsest_fp32=flag,
                         precision=amg.AMG_FP32_IN_FP64)
        try:
            z = solver.vcycle(torch.from_numpy(b).cuda())
            torch.cuda.synchronize()
            errs.append(np.abs(z.cpu().numpy() - ref).max() / np.abs(ref).max())
        finally:
            solver.close()
    # float32 unit roundoff 6e-8 times n terms and cond(M)
    bound = n * 6e-8 * np.linalg.cond(M)
    assert errs[0] <= bound and errs[1] <= bound
    assert errs[1] > 0.0


@pytest.mark.parametrize("flex", [0, 1])
def test_float32_coarsest_inverse_converges(flex):
    p = P.lognormal3d((28, 24, 20), seed=3)
    b = torch.from_numpy(p.b).cuda()
    its = []
    for flag in (0, 1):
        solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, coarsest_fp32=flag,
                         precision=amg.AMG_FP32_IN_FP64, flexible_cg=flex)
        try:
            x, rc, info = solver.solve(b, tol=1e-8, maxit=300)
            assert rc == amg.AMG_OK and info["true_rel_residual"] <= 1.05e-8
            its.append(info["iterations"])
        finally:
            solver.close()
    assert abs(its[0] - its[1]) <= 1
