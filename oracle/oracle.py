"""ctypes wrapper around the C++ oracle (amg_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the benchmark's CPU-baseline leg.  The library under test never imports
this module, and this module never imports the library.

All functions take plain numpy arrays (int32 CSR indices, float64 values) in
the original row numbering of the matrix.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lib = None
_lib_omp = None

# Default parameters of the reading documented in the oracle source:
# delta = 1/3, beta = 1e-5, omega = 1.6, s_min = 2^d, s_max = 3 * 2^(d-1),
# d_max = d, coarsening target 5000 rows, at most 20 levels, dense coarsest
# solve up to 8192 rows, stop when n_l / n_{l+1} < 1.2.
def default_params(dim: int) -> dict:
    return dict(delta=1.0 / 3.0, beta=1e-5, omega=1.6,
                s_min=2 ** dim, s_max=3 * 2 ** (dim - 1), d_max=dim,
                coarsen_target=5000, max_levels=20, dense_cap=8192, min_rate=1.2,
                smoother=0)


_ORDER = ["delta", "beta", "omega", "s_min", "s_max", "d_max",
          "coarsen_target", "max_levels", "dense_cap", "min_rate", "smoother", "agg_tile"]


def _param_array(p: dict) -> np.ndarray:
    # smoother: 0 multicolour symmetric GS (the GPU's order), 1 sequential
    # symmetric GS in index order; agg_tile: > 0 decoupled aggregation in
    # tiles of that many consecutive rows (Alg. 4), 0 one sequential pass
    return np.array([float(p.get(k, 0)) for k in _ORDER], dtype=np.float64)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, plain -O2); openmp:
    the same source with -fopenmp, for the CPU baseline on all host cores."""
    out = _OUT_OMP if openmp else _OUT
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC",
                               *flags, "-shared", _SRC, "-o", tmp])
        os.replace(tmp, out)
    return out


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if (_lib_omp if openmp else _lib) is not None:
        return _lib_omp if openmp else _lib
    lib = ctypes.CDLL(build(openmp=openmp))
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    lib.oracle_strength.argtypes = [I, P, P, P, P, P, P, P, P]
    lib.oracle_aggregate.argtypes = [I, P, P, P, P, P]
    lib.oracle_aggregate.restype = I
    lib.oracle_colour.argtypes = [I, P, P, P, I]
    lib.oracle_colour.restype = I
    lib.oracle_galerkin.argtypes = [I, P, P, P, P, I, P, P, P]
    lib.oracle_galerkin.restype = I
    lib.oracle_spmv.argtypes = [I, P, P, P, P, P]
    lib.oracle_setup.argtypes = [I, P, P, P, P, P]
    lib.oracle_setup.restype = P
    lib.oracle_num_levels.argtypes = [P]
    lib.oracle_num_levels.restype = I
    lib.oracle_level_info.argtypes = [P, I, P]
    lib.oracle_level_export.argtypes = [P, I, P, P, P, P, P]
    lib.oracle_vcycle.argtypes = [P, P, P]
    lib.oracle_pcg.argtypes = [P, P, P, D, I, I, P]
    lib.oracle_pcg.restype = I
    lib.oracle_bicgstab.argtypes = [P, P, P, D, I, P]
    lib.oracle_bicgstab.restype = I
    lib.oracle_free.argtypes = [P]
    lib.oracle_threads.argtypes = [I]
    lib.oracle_threads.restype = I
    if openmp:
        _lib_omp = lib
    else:
        _lib = lib
    return lib


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the thread count of the OpenMP build."""
    return int(_load(openmp=True).oracle_threads(int(n)))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(rp, ci, va):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    va = np.ascontiguousarray(va, dtype=np.float64)
    return rp, ci, va


def strength(rp, ci, va, params: dict):
    """Returns (eta_max, isolated, dirichlet, strong-per-entry)."""
    rp, ci, va = _csr(rp, ci, va)
    n = rp.shape[0] - 1
    eta = np.zeros(n)
    iso = np.zeros(n, dtype=np.int8)
    dirich = np.zeros(n, dtype=np.int8)
    strong = np.zeros(ci.shape[0], dtype=np.int8)
    pa = _param_array(params)
    _load().oracle_strength(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(pa), _ptr(eta),
                            _ptr(iso), _ptr(dirich), _ptr(strong))
    return eta, iso.astype(bool), dirich.astype(bool), strong.astype(bool)


def aggregate(rp, ci, va, params: dict):
    """Algorithm 1 on the matrix graph; returns (agg, n_coarse)."""
    rp, ci, va = _csr(rp, ci, va)
    n = rp.shape[0] - 1
    agg = np.zeros(n, dtype=np.int32)
    pa = _param_array(params)
    nc = _load().oracle_aggregate(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(pa), _ptr(agg))
    return agg, int(nc)


COLOUR_SMOOTHER, COLOUR_GREEDY, COLOUR_DSATUR = 0, 1, 2


def colour(rp, ci, method: int = COLOUR_SMOOTHER):
    """Colouring of the matrix graph: the smoother's (fewer colours of the
    two below), ascending-order greedy, or DSATUR."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    n = rp.shape[0] - 1
    c = np.zeros(n, dtype=np.int32)
    nc = _load().oracle_colour(n, _ptr(rp), _ptr(ci), _ptr(c), int(method))
    return c, int(nc)


def galerkin(rp, ci, va, agg, nc: int):
    """G = P^T A P as CSR (row_ptr, col, val)."""
    rp, ci, va = _csr(rp, ci, va)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    n = rp.shape[0] - 1
    lib = _load()
    nnz = lib.oracle_galerkin(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(agg), nc, None, None, None)
    grp = np.zeros(nc + 1, dtype=np.int32)
    gci = np.zeros(nnz, dtype=np.int32)
    gva = np.zeros(nnz)
    lib.oracle_galerkin(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(agg), nc, _ptr(grp), _ptr(gci), _ptr(gva))
    return grp, gci, gva


def spmv(rp, ci, va, x):
    rp, ci, va = _csr(rp, ci, va)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(rp.shape[0] - 1)
    _load().oracle_spmv(rp.shape[0] - 1, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x), _ptr(y))
    return y


class Hierarchy:
    """The oracle's AMG hierarchy for one matrix."""

    def __init__(self, rp, ci, va, params: dict, openmp: bool = False):
        """openmp: run on the OpenMP build of the same source (CPU baseline
        on all cores; see threads())."""
        rp, ci, va = _csr(rp, ci, va)
        self.n = rp.shape[0] - 1
        self._keep = (rp, ci, va)
        pa = _param_array(params)
        st = ctypes.c_int(0)
        self._lib = _load(openmp)
        self._h = self._lib.oracle_setup(self.n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(pa),
                                         ctypes.byref(st))
        self.status = st.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_free(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return self._lib.oracle_num_levels(self._h)

    def level(self, l: int) -> dict:
        info = np.zeros(4, dtype=np.int32)
        self._lib.oracle_level_info(self._h, l, _ptr(info))
        n, nnz, nc, ncol = (int(v) for v in info)
        rp = np.zeros(n + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        va = np.zeros(nnz)
        agg = np.full(n, -1, dtype=np.int32)
        col = np.full(n, -1, dtype=np.int32)
        self._lib.oracle_level_export(self._h, l, _ptr(rp), _ptr(ci), _ptr(va), _ptr(agg), _ptr(col))
        last = l == self.num_levels - 1
        return dict(n=n, nnz=nnz, nc=nc, ncolours=ncol, row_ptr=rp, col=ci, val=va,
                    agg=None if last else agg, colour=None if last else col)

    def vcycle(self, r: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros(self.n)
        self._lib.oracle_vcycle(self._h, _ptr(r), _ptr(z))
        return z

    def pcg(self, b: np.ndarray, tol: float = 1e-8, maxit: int = 500,
            x0: Optional[np.ndarray] = None, flexible: bool = False):
        """Returns (x, iterations or negative status, recursive rel. residual,
        true rel. residual)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        out = np.zeros(2)
        it = self._lib.oracle_pcg(self._h, _ptr(b), _ptr(x), float(tol), int(maxit),
                                  int(bool(flexible)), _ptr(out))
        return x, int(it), float(out[0]), float(out[1])

    def bicgstab(self, b: np.ndarray, tol: float = 1e-8, maxit: int = 500,
                 x0: Optional[np.ndarray] = None):
        """Preconditioned BiCGSTAB (Sec. 5).  Returns (x, iterations or
        negative status, recursive rel. residual, true rel. residual,
        V-cycles applied)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        out = np.zeros(3)
        it = self._lib.oracle_bicgstab(self._h, _ptr(b), _ptr(x), float(tol), int(maxit), _ptr(out))
        return x, int(it), float(out[0]), float(out[1]), int(out[2])
