import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: full-size workloads")


def _has_cuda() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_cuda():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


# ---------------------------------------------------------------------------
# small matrices shared by the tests
# ---------------------------------------------------------------------------

def const_diag_grid(shape, diag):
    """diag * I - adjacency of a structured grid (x fastest)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[:a])) for a in range(len(shape))]
    rows, cols, vals = [], [], []
    for idx in range(n):
        co = [(idx // strides[a]) % shape[a] for a in range(len(shape))]
        ent = [(idx, float(diag))]
        for a in range(len(shape)):
            if co[a] > 0:
                ent.append((idx - strides[a], -1.0))
            if co[a] < shape[a] - 1:
                ent.append((idx + strides[a], -1.0))
        for j, v in sorted(ent):
            rows.append(idx); cols.append(j); vals.append(v)
    return coo_to_csr(n, rows, cols, vals)


def weighted_path(weights, end_shift):
    """Path graph with the given edge weights; diagonal = sum of incident
    weights, plus ``end_shift`` on the two end vertices."""
    n = len(weights) + 1
    rows, cols, vals = [], [], []
    for i in range(n):
        d = 0.0
        ent = []
        if i > 0:
            ent.append((i - 1, -weights[i - 1])); d += weights[i - 1]
        if i < n - 1:
            ent.append((i + 1, -weights[i])); d += weights[i]
        if i == 0 or i == n - 1:
            d += end_shift
        ent.append((i, d))
        for j, v in sorted(ent):
            rows.append(i); cols.append(j); vals.append(v)
    return coo_to_csr(n, rows, cols, vals)


def coo_to_csr(n, rows, cols, vals):
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int32)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp).astype(np.int32), cols, vals


def graph_from_spec(spec):
    kind = spec["kind"]
    if kind == "const_diag_grid":
        return const_diag_grid(spec["shape"], spec["diag"])
    if kind == "weighted_path":
        return weighted_path(spec["weights"], spec["end_shift"])
    if kind == "explicit":
        e = spec["entries"]
        return coo_to_csr(spec["n"], [t[0] for t in e], [t[1] for t in e], [t[2] for t in e])
    raise KeyError(kind)


def to_dense(rp, ci, va):
    n = len(rp) - 1
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i, ci[k]] += va[k]
    return A


def oracle_iterate(H, b, it_gpu, it_o, xo, x0=None):
    """The oracle's CG iterate after the GPU's iteration count.  The bar on
    iterations (within 1) lets the two stop one step apart, and the step
    between them can exceed the solution bar on badly conditioned problems,
    so solutions are compared at the same step."""
    if it_gpu == it_o:
        return xo
    x, _, _, _ = H.pcg(b, tol=1e-300, maxit=it_gpu, x0=x0)
    return x
