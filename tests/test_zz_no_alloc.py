"""The allocation-free residual norm (amg_residual_norm_noalloc).

Some callers cannot allocate device memory where they need a residual check:
a loop sharing the GPU with other streams cannot afford the device-wide
synchronisation cudaMalloc may cause, an allocator hook must not re-enter the
allocator, and a program whose memory belongs to a pool it does not control has
nothing to allocate from.  The allocation-free entry point serves them and must
give the same norm as the context-based amg_residual_norm, and the norm that
numpy computes from the oracle's SpMV.  This file is collected last, so a failure
here comes after every other test has run; it passes both on its own in a fresh
process and after the rest of the suite."""

import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12   # relative, as the other float64 norm checks of the suite


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_residual_norm_matches_the_context_entry_point_on_two_calls():
    p = P.lognormal3d((40, 36, 33), seed=2)
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3)
    rp, ci, va, b = _dev(p.row_ptr), _dev(p.col), _dev(p.val), _dev(p.b)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(11)
    for _ in range(2):   # two calls in a row share the scratch array
        xh = rng.standard_normal(p.n)
        x = _dev(xh)
        ref = solver.residual_norm(b, x)
        amg.amg_residual_norm_noalloc(rp, ci, va, b, x, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= TOL * ref, (got, ref)
        # and against a norm formed without the library: the oracle's SpMV, numpy
        ind = np.linalg.norm(p.b - O.spmv(p.row_ptr, p.col, p.val, xh))
        assert abs(got - ind) <= TOL * ind, (got, ind)
    solver.close()


def test_noalloc_residual_norm_at_its_row_limit():
    # n = 16,777,216 rows: the largest the fixed scratch takes, a grid of
    # 65,536 blocks whose partial sums fill the array; a diagonal matrix keeps
    # the reference a plain numpy expression
    n = 16_777_216
    rng = np.random.default_rng(5)
    d = 1.0 + rng.random(n)
    bh = rng.standard_normal(n)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rp = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.arange(n, dtype=torch.int32, device="cuda")
    va, b = _dev(d), _dev(bh)
    for seed in (1, 2):
        xh = np.random.default_rng(seed).standard_normal(n)
        amg.amg_residual_norm_noalloc(rp, ci, va, b, _dev(xh), out)
        torch.cuda.synchronize()
        ref = float(np.linalg.norm(bh - d * xh))
        got = float(out.item())
        assert abs(got - ref) <= TOL * ref, (got, ref)


def test_noalloc_residual_norm_rejects_matrices_beyond_its_scratch():
    tiny_i = torch.zeros(4, dtype=torch.int32, device="cuda")
    tiny_d = torch.zeros(4, dtype=torch.float64, device="cuda")
    A = amg.amg_csr(16_777_217, 1, tiny_i.data_ptr(), tiny_i.data_ptr(), tiny_d.data_ptr(), 1)
    rc = amg.lib().amg_residual_norm_noalloc(ctypes.byref(A), tiny_d.data_ptr(),
                                             tiny_d.data_ptr(), tiny_d.data_ptr(), None)
    assert rc == amg.AMG_EINVAL
    assert "16777216" in amg.amg_last_error()


def test_noalloc_residual_norm_rejects_host_pointers_before_launch():
    # a host vector among device ones is refused by the library itself (the
    # pointer query), and the device output keeps its old value
    p = P.laplace2d_random_rhs(16, seed=0)
    rp, ci, va, b = _dev(p.row_ptr), _dev(p.col), _dev(p.val), _dev(p.b)
    out = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    xh = np.zeros(p.n)
    A = amg.amg_csr(p.n, p.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1)
    for bad in ("b", "x", "norm"):
        args = {"b": b.data_ptr(), "x": _dev(xh).data_ptr(), "norm": out.data_ptr()}
        host = np.zeros(max(1, p.n)) if bad != "norm" else np.zeros(1)
        args[bad] = host.ctypes.data
        rc = amg.lib().amg_residual_norm_noalloc(ctypes.byref(A), args["b"], args["x"],
                                                 args["norm"], None)
        assert rc == amg.AMG_EINVAL, bad
        assert "device memory" in amg.amg_last_error()
    torch.cuda.synchronize()
    assert float(out.item()) == -7.0
