"""The checked build (libamg_checked.so, compiled with AMG_DEVICE_CHECKS):
every solve kernel tests each index it gathers against its range and records
AMG_ERANGE instead of reading out of range.  It stands in for a memory
sanitizer on this GPU.  Each test runs in a child process that loads the
checked library (AMG_LIB=checked), so the rest of the suite keeps the regular
one.  Also: both builds stop a Krylov solve whose dot products turn
non-finite."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from oracle import oracle as O
from paper_1209_0960_gb300 import amg, problems as P
assert amg.lib().amg_device_checks() == 1
torch.cuda.set_device(0)
out = {}
cases = {
    "lognormal": (lambda: P.lognormal3d((28, 24, 20), seed=1), {"coarsen_target": 300}),
    "layered": (lambda: P.layered3d((20, 20, 24), seed=3), {"coarsen_target": 200}),
    "hub": (lambda: P.hub_graph2d(48), {"coarsen_target": 100}),
    "aniso_48": (lambda: P.anisotropic3d((48, 48, 48), seed=0), {}),
}
for name, (mk, over) in cases.items():
    p = mk()
    s = amg.AMG(p.row_ptr, p.col, p.val, dim=p.dim, autotune=1, **over)
    b = torch.from_numpy(p.b).cuda()
    res = []
    for prec in (amg.AMG_FP64, amg.AMG_FP32_IN_FP64):
        s.set_precision(prec)
        x, rc, info = s.solve(b, tol=1e-10 if prec == amg.AMG_FP64 else 1e-8, maxit=400)
        r = p.b - O.spmv(p.row_ptr, p.col, p.val, x.cpu().numpy())
        res.append([rc, info["iterations"], float(np.linalg.norm(r) / np.linalg.norm(p.b))])
    x, rc, info = s.solve_bicgstab(b, tol=1e-10, maxit=400)
    res.append([rc, info["iterations"], info["true_rel_residual"]])
    out[name] = res
    s.close()
# a corrupt hierarchy: one stored column index of level 1 set past the level's
# rows (an index no kernel of either build dereferences); the checks report it
p = P.lognormal3d((28, 24, 20), seed=1)
s = amg.AMG(p.row_ptr, p.col, p.val, dim=3, coarsen_target=300)
b = torch.from_numpy(p.b).cuda()
lev = s.info()[1]
n1 = lev[1]["n"]
rc = amg.lib().amg_debug_set_column(s.ctx, 1, 5, 0, n1 + 3)
out["poke"] = rc
x, rc, info = s.solve(b, tol=1e-10, maxit=50)
out["corrupt_solve"] = [rc, amg.amg_last_error()]
# the same entry read by the staged kernels from the level's compact copy
s.set_level_shape(1, 0)
out["staged_compact"] = s.info()[1][1]["compact"]
x, rc, info = s.solve(b, tol=1e-10, maxit=50)
out["corrupt_solve_staged"] = [rc, amg.amg_last_error()]
s.close()
print("RESULT " + json.dumps(out))
"""


def _run_child():
    env = dict(os.environ, AMG_LIB="checked")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def checked():
    from paper_1209_0960_gb300 import build as B
    B.build(checked=True)
    return _run_child()


def test_checked_build_solves_every_workload_without_a_range_report(checked):
    # the checks raise no alarm on valid hierarchies (every launch shape the
    # tuner picks, both precisions, PCG and BiCGSTAB)
    for name in ("lognormal", "layered", "hub", "aniso_48"):
        (rc64, it64, res64), (rc32, it32, res32), (rcb, itb, resb) = checked[name]
        assert rc64 == amg.AMG_OK and res64 <= 1.5e-10, name
        assert rc32 == amg.AMG_OK and res32 <= 1.05e-8, name
        assert rcb == amg.AMG_OK and resb <= 1.5e-10, name


def test_checked_build_matches_the_regular_build(checked):
    # the checks change no arithmetic: same iteration counts as the regular build
    p = P.lognormal3d((28, 24, 20), seed=1)
    s = amg.AMG(p.row_ptr, p.col, p.val, dim=3, autotune=1, coarsen_target=300)
    try:
        x, rc, info = s.solve(torch.from_numpy(p.b).cuda(), tol=1e-10, maxit=400)
        assert rc == amg.AMG_OK and info["iterations"] == checked["lognormal"][0][1]
    finally:
        s.close()


def test_checked_build_reports_a_corrupt_index(checked):
    assert checked["poke"] == amg.AMG_OK
    rc, msg = checked["corrupt_solve"]
    assert rc == amg.AMG_ERANGE
    assert "outside its range" in msg
    assert checked["staged_compact"] == 1
    rc, msg = checked["corrupt_solve_staged"]
    assert rc == amg.AMG_ERANGE
    assert "outside its range" in msg


def test_non_finite_dot_products_stop_the_solve():
    # a NaN in the right-hand side makes ||r_0|| NaN: PCG and BiCGSTAB stop
    # with AMG_ENONFINITE instead of iterating to maxit or reporting success
    p = P.lognormal3d((16, 16, 16), seed=2)
    s = amg.AMG(p.row_ptr, p.col, p.val, dim=3)
    try:
        bh = p.b.copy()
        bh[7] = np.nan
        b = torch.from_numpy(bh).cuda()
        for loop in (1, 0):
            x, rc, info = s.solve(b, tol=1e-8, maxit=50)
            assert rc == amg.AMG_ENONFINITE
            assert info["iterations"] == 0
        x, rc, info = s.solve_bicgstab(b, tol=1e-8, maxit=50)
        assert rc == amg.AMG_ENONFINITE
        assert "not finite" in amg.amg_last_error()
        # the context stays usable
        x, rc, info = s.solve(torch.from_numpy(p.b).cuda(), tol=1e-8)
        assert rc == amg.AMG_OK
    finally:
        s.close()
