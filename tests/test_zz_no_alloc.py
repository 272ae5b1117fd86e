"""The allocation-free residual norm (amg_residual_norm_noalloc) against the
context-based amg_residual_norm.

Callers that cannot allocate device memory when they need a residual check --
for example code running during CUDA graph capture -- use the allocation-free
entry point; it must give the same norm as the regular one.  This file is
collected last, so a failure here comes after every other test has run, and it
passes both on its own in a fresh process and after the rest of the suite."""

import numpy as np
import pytest

from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_residual_norm_matches_the_context_entry_point_on_two_calls():
    p = P.lognormal3d((40, 36, 33), seed=2)
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3)
    rp = torch.from_numpy(p.row_ptr).cuda()
    ci = torch.from_numpy(p.col).cuda()
    va = torch.from_numpy(p.val).cuda()
    b = torch.from_numpy(p.b).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(11)
    for _ in range(2):   # two calls in a row share the scratch array
        x = torch.from_numpy(rng.standard_normal(p.n)).cuda()
        ref = solver.residual_norm(b, x)
        amg.amg_residual_norm_noalloc(rp, ci, va, b, x, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    solver.close()


def test_noalloc_residual_norm_rejects_matrices_beyond_its_scratch():
    tiny_i = torch.zeros(4, dtype=torch.int32, device="cuda")
    tiny_d = torch.zeros(4, dtype=torch.float64, device="cuda")
    A = amg.amg_csr(16_777_217, 1, tiny_i.data_ptr(), tiny_i.data_ptr(), tiny_d.data_ptr(), 1)
    rc = amg.lib().amg_residual_norm_noalloc(amg.ctypes.byref(A), tiny_d.data_ptr(),
                                             tiny_d.data_ptr(), tiny_d.data_ptr(), None)
    assert rc == amg.AMG_EINVAL
    assert "16777216" in amg.amg_last_error()
