"""Thin ctypes binding of libamg (include/amg.h).

Every function named ``amg_*`` here forwards to the C entry point of the same
name; the binding only marshals arguments (numpy arrays for host buffers,
torch CUDA tensors for device buffers) and turns negative return codes into
``AmgError``.  All computation happens in the CUDA library: if it is not built,
``lib()`` raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

AMG_OK = 0
AMG_PENDING = 1
AMG_EINVAL = -1
AMG_ENOMEM = -2
AMG_ENOTSPD = -3
AMG_ENOTCONV = -4
AMG_ETIMEOUT = -5
AMG_ECUDA = -6
AMG_ENOTFOUND = -7
AMG_ERANGE = -8
AMG_ENONFINITE = -9

# statuses a solve returns together with its info record (not raised)
_SOLVE_STATUSES = (AMG_ENOTCONV, AMG_ENOTSPD, AMG_ENONFINITE, AMG_ERANGE, AMG_ETIMEOUT)

AMG_FP64 = 0
AMG_FP32_IN_FP64 = 1
AMG_SHAPE_SWEEP = 0x100   # or'ed into lanes_per_row: one dependency-driven kernel per sweep

_c_i32 = ctypes.c_int32
_c_dbl = ctypes.c_double
_c_vp = ctypes.c_void_p


class amg_csr(ctypes.Structure):
    _fields_ = [("n", _c_i32), ("nnz", _c_i32), ("row_ptr", _c_vp), ("col", _c_vp),
                ("val", _c_vp), ("on_device", _c_i32)]


class amg_params(ctypes.Structure):
    _fields_ = [("delta", _c_dbl), ("beta", _c_dbl), ("omega", _c_dbl),
                ("s_min", _c_i32), ("s_max", _c_i32), ("d_max", _c_i32),
                ("coarsen_target", _c_i32), ("max_levels", _c_i32), ("dense_cap", _c_i32),
                ("min_coarsen_rate", _c_dbl), ("precision", _c_i32), ("flexible_cg", _c_i32),
                ("cuda_stream", _c_vp), ("launch_overlap", _c_i32),
                ("aggregation_tile", _c_i32), ("aggregation_device", _c_i32),
                ("host_threads", _c_i32), ("coarsest_fp32", _c_i32), ("device_loop", _c_i32),
                ("autotune", _c_i32)]


class amg_solve_info(ctypes.Structure):
    _fields_ = [("status", _c_i32), ("iterations", _c_i32), ("rel_residual", _c_dbl),
                ("true_rel_residual", _c_dbl), ("solve_ms", _c_dbl), ("device_loop", _c_i32)]


class amg_level_info(ctypes.Structure):
    _fields_ = [("n", _c_i32), ("nnz", _c_i32), ("n_coarse", _c_i32), ("ncolours", _c_i32),
                ("max_agg_size", _c_i32), ("n_isolated", _c_i32), ("n_dirichlet", _c_i32),
                ("vcycle_bytes_fp64", _c_dbl), ("vcycle_bytes_fp32", _c_dbl),
                ("lanes_per_row", _c_i32), ("threads_per_block", _c_i32), ("sweep", _c_i32),
                ("compact", _c_i32), ("staged_entries", ctypes.c_int64), ("carveout", _c_i32)]


class amg_summary(ctypes.Structure):
    _fields_ = [("num_levels", _c_i32), ("coarsest_n", _c_i32),
                ("operator_complexity", _c_dbl), ("host_setup_ms", _c_dbl),
                ("gpu_galerkin_ms", _c_dbl), ("gpu_other_ms", _c_dbl), ("total_setup_ms", _c_dbl),
                ("vcycle_bytes_fp64", _c_dbl), ("vcycle_bytes_fp32", _c_dbl),
                ("pcg_iter_bytes_fp64", _c_dbl), ("pcg_iter_bytes_fp32", _c_dbl),
                ("aggregation_ms", _c_dbl), ("autotune_ms", _c_dbl),
                ("coarsest_inverse_ms", _c_dbl)]


class amg_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _c_i32), ("total_ms", _c_dbl),
                ("bytes", _c_dbl)]


class amg_server_params(ctypes.Structure):
    _fields_ = [("params", amg_params), ("max_slots", _c_i32), ("setup_threads", _c_i32),
                ("maxit", _c_i32), ("hbm_budget_bytes", _c_dbl), ("batch_vcycles", _c_i32)]


class amg_request_times(ctypes.Structure):
    _fields_ = [("queue_ms", _c_dbl), ("setup_ms", _c_dbl), ("solve_ms", _c_dbl),
                ("total_ms", _c_dbl), ("hbm_bytes", _c_dbl)]


class amg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", _c_i32), ("running", _c_i32),
                ("peak_running", _c_i32), ("hbm_reserved_bytes", _c_dbl),
                ("hbm_budget_bytes", _c_dbl), ("batched_vcycles", ctypes.c_int64),
                ("batched_requests", ctypes.c_int64)]


def struct_dict(s) -> dict:
    return {name: getattr(s, name) for name, _ in s._fields_}


class AmgError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


# exported symbols and their signatures, as declared in include/amg.h
_SIGNATURES = {
    "amg_params_default": ([ctypes.POINTER(amg_params), _c_i32], ctypes.c_int),
    "amg_setup": ([ctypes.POINTER(amg_csr), ctypes.POINTER(amg_params), ctypes.POINTER(_c_vp)], ctypes.c_int),
    "amg_set_precision": ([_c_vp, _c_i32, _c_i32], ctypes.c_int),
    "amg_vcycle": ([_c_vp, _c_vp, _c_vp], ctypes.c_int),
    "amg_pcg_solve": ([_c_vp, _c_vp, _c_vp, _c_dbl, _c_i32, ctypes.POINTER(amg_solve_info)], ctypes.c_int),
    "amg_bicgstab_solve": ([_c_vp, _c_vp, _c_vp, _c_dbl, _c_i32, ctypes.POINTER(amg_solve_info)], ctypes.c_int),
    "amg_pcg_solve_host": ([_c_vp, _c_vp, _c_vp, _c_dbl, _c_i32, ctypes.POINTER(amg_solve_info)], ctypes.c_int),
    "amg_pcg_solve_host_zero_guess": ([_c_vp, _c_vp, _c_vp, _c_dbl, _c_i32, ctypes.POINTER(amg_solve_info)],
                                      ctypes.c_int),
    "amg_residual_norm": ([_c_vp, _c_vp, _c_vp, ctypes.POINTER(_c_dbl)], ctypes.c_int),
    "amg_residual_norm_noalloc": ([ctypes.POINTER(amg_csr), _c_vp, _c_vp, _c_vp, _c_vp], ctypes.c_int),
    "amg_hierarchy_info": ([_c_vp, ctypes.POINTER(amg_summary), ctypes.POINTER(amg_level_info), _c_i32], ctypes.c_int),
    "amg_export_level": ([_c_vp, _c_i32, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp], ctypes.c_int),
    "amg_set_level_shape": ([_c_vp, _c_i32, _c_i32, _c_i32], ctypes.c_int),
    "amg_set_level_carveout": ([_c_vp, _c_i32, _c_i32], ctypes.c_int),
    "amg_selftest_bounded_wait": ([ctypes.c_int64, _c_vp, ctypes.POINTER(_c_i32),
                                   ctypes.POINTER(_c_dbl)], ctypes.c_int),
    "amg_aggregate": ([ctypes.POINTER(amg_csr), ctypes.POINTER(amg_params), _c_vp, ctypes.POINTER(_c_i32)], ctypes.c_int),
    "amg_colour": ([ctypes.POINTER(amg_csr), _c_vp, ctypes.POINTER(_c_i32)], ctypes.c_int),
    "amg_profile_enable": ([_c_vp, _c_i32], ctypes.c_int),
    "amg_profile_read": ([_c_vp, ctypes.POINTER(amg_kernel_stat), _c_i32], ctypes.c_int),
    "amg_free": ([_c_vp], ctypes.c_int),
    "amg_server_params_default": ([ctypes.POINTER(amg_server_params), _c_i32], ctypes.c_int),
    "amg_server_create": ([ctypes.POINTER(amg_server_params), ctypes.POINTER(_c_vp)], ctypes.c_int),
    "amg_submit": ([_c_vp, ctypes.POINTER(amg_csr), _c_vp, _c_dbl, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "amg_poll": ([_c_vp, ctypes.c_uint64, _c_vp, ctypes.POINTER(amg_solve_info),
                  ctypes.POINTER(amg_request_times)], ctypes.c_int),
    "amg_server_stats_read": ([_c_vp, ctypes.POINTER(amg_server_stats)], ctypes.c_int),
    "amg_server_destroy": ([_c_vp], ctypes.c_int),
    "amg_last_error": ([], ctypes.c_char_p),
    "amg_device_checks": ([], ctypes.c_int),
    "amg_debug_set_column": ([_c_vp, _c_i32, _c_i32, _c_i32, _c_i32], ctypes.c_int),
}

_lib = None


def lib_path() -> str:
    """libamg.so, or libamg_checked.so (the build whose kernels test every
    index they gather) when the environment sets AMG_LIB=checked."""
    return _build.LIB_CHECKED if os.environ.get("AMG_LIB", "") == "checked" else _build.LIB


def lib(build_if_missing: bool = False):
    """The loaded library (see lib_path).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        _build.build(checked=path == _build.LIB_CHECKED)
    if not os.path.exists(path):
        raise RuntimeError(f"libamg.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc: int, where: str, allow=()):
    if rc < 0 and rc not in allow:
        msg = lib().amg_last_error()
        raise AmgError(rc, where, msg.decode() if msg else "")
    return rc


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (None passes through)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return int(a.data_ptr())


# ---------------------------------------------------------------------------
# entry points, same names as the C ABI
# ---------------------------------------------------------------------------

def amg_params_default(dim: int) -> amg_params:
    p = amg_params()
    _check(lib().amg_params_default(ctypes.byref(p), dim), "amg_params_default")
    return p


def amg_setup(row_ptr, col, val, params: amg_params) -> int:
    """row_ptr/col/val: numpy (host) or torch CUDA tensors (device)."""
    on_dev = not isinstance(row_ptr, np.ndarray)
    if not on_dev:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
    n = int(row_ptr.shape[0]) - 1
    A = amg_csr(n, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val), int(on_dev))
    h = _c_vp()
    _check(lib().amg_setup(ctypes.byref(A), ctypes.byref(params), ctypes.byref(h)), "amg_setup")
    return h.value


def amg_set_precision(ctx: int, precision: int, flexible_cg: int = -1) -> None:
    _check(lib().amg_set_precision(ctx, precision, flexible_cg), "amg_set_precision")


def amg_vcycle(ctx: int, r_dev, z_dev) -> None:
    _check(lib().amg_vcycle(ctx, _ptr(r_dev), _ptr(z_dev)), "amg_vcycle")


def amg_pcg_solve(ctx: int, b_dev, x_dev, tol: float, maxit: int):
    info = amg_solve_info()
    rc = lib().amg_pcg_solve(ctx, _ptr(b_dev), _ptr(x_dev), tol, maxit, ctypes.byref(info))
    _check(rc, "amg_pcg_solve", allow=_SOLVE_STATUSES)
    return rc, info


def amg_bicgstab_solve(ctx: int, b_dev, x_dev, tol: float, maxit: int):
    info = amg_solve_info()
    rc = lib().amg_bicgstab_solve(ctx, _ptr(b_dev), _ptr(x_dev), tol, maxit, ctypes.byref(info))
    _check(rc, "amg_bicgstab_solve", allow=_SOLVE_STATUSES)
    return rc, info


def amg_pcg_solve_host(ctx: int, b_host: np.ndarray, x_host: np.ndarray, tol: float, maxit: int):
    info = amg_solve_info()
    rc = lib().amg_pcg_solve_host(ctx, _ptr(b_host), _ptr(x_host), tol, maxit, ctypes.byref(info))
    _check(rc, "amg_pcg_solve_host", allow=_SOLVE_STATUSES)
    return rc, info


def amg_pcg_solve_host_zero_guess(ctx: int, b_host: np.ndarray, x_host: np.ndarray, tol: float,
                                  maxit: int):
    info = amg_solve_info()
    rc = lib().amg_pcg_solve_host_zero_guess(ctx, _ptr(b_host), _ptr(x_host), tol, maxit,
                                             ctypes.byref(info))
    _check(rc, "amg_pcg_solve_host_zero_guess", allow=_SOLVE_STATUSES)
    return rc, info


def amg_residual_norm(ctx: int, b_dev, x_dev) -> float:
    out = _c_dbl()
    _check(lib().amg_residual_norm(ctx, _ptr(b_dev), _ptr(x_dev), ctypes.byref(out)),
           "amg_residual_norm")
    return out.value


def amg_residual_norm_noalloc(row_ptr_dev, col_dev, val_dev, b_dev, x_dev, norm_dev,
                              stream=None) -> None:
    """||b - A x|| into the device tensor norm_dev (one float64) without any
    allocation; A given as device CSR tensors (int32, int32, float64).
    Raises ValueError for CPU tensors, other dtypes or non-contiguous tensors
    before the library is called (the library itself rejects host pointers
    with AMG_EINVAL)."""
    want = (("row_ptr_dev", row_ptr_dev, "int32"), ("col_dev", col_dev, "int32"),
            ("val_dev", val_dev, "float64"), ("b_dev", b_dev, "float64"),
            ("x_dev", x_dev, "float64"), ("norm_dev", norm_dev, "float64"))
    devs = set()
    for name, t, dt in want:
        if isinstance(t, np.ndarray) or not getattr(t, "is_cuda", False):
            raise ValueError(f"amg_residual_norm_noalloc: {name} must be a CUDA tensor")
        if str(t.dtype).replace("torch.", "") != dt:
            raise ValueError(f"amg_residual_norm_noalloc: {name} must be {dt}, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"amg_residual_norm_noalloc: {name} must be contiguous")
        devs.add(t.device)
    if len(devs) != 1:
        raise ValueError("amg_residual_norm_noalloc: all tensors must be on one device")
    n = int(row_ptr_dev.shape[0]) - 1
    if b_dev.numel() != n or x_dev.numel() != n or norm_dev.numel() < 1 or val_dev.numel() != col_dev.numel():
        raise ValueError("amg_residual_norm_noalloc: inconsistent sizes")
    A = amg_csr(n, int(col_dev.shape[0]), _ptr(row_ptr_dev), _ptr(col_dev), _ptr(val_dev), 1)
    s = None if stream is None else int(stream.cuda_stream)
    _check(lib().amg_residual_norm_noalloc(ctypes.byref(A), _ptr(b_dev), _ptr(x_dev), _ptr(norm_dev), s),
           "amg_residual_norm_noalloc")


def amg_hierarchy_info(ctx: int):
    s = amg_summary()
    nl = _check(lib().amg_hierarchy_info(ctx, ctypes.byref(s), None, 0), "amg_hierarchy_info")
    levels = (amg_level_info * nl)()
    _check(lib().amg_hierarchy_info(ctx, ctypes.byref(s), levels, nl), "amg_hierarchy_info")
    return struct_dict(s), [struct_dict(l) for l in levels]


def amg_selftest_bounded_wait(polls: int, stream=None):
    """Returns (status recorded by the kernel, kernel milliseconds)."""
    st = _c_i32(0)
    ms = _c_dbl(0.0)
    _check(lib().amg_selftest_bounded_wait(int(polls), stream, ctypes.byref(st), ctypes.byref(ms)),
           "amg_selftest_bounded_wait")
    return st.value, ms.value


def amg_set_level_shape(ctx: int, l: int, lanes_per_row: int, threads_per_block: int = 0) -> None:
    _check(lib().amg_set_level_shape(ctx, l, lanes_per_row, threads_per_block),
           "amg_set_level_shape")


def amg_set_level_carveout(ctx: int, l: int, percent: int) -> None:
    _check(lib().amg_set_level_carveout(ctx, l, percent), "amg_set_level_carveout")


def amg_export_level(ctx: int, l: int) -> dict:
    _, levels = amg_hierarchy_info(ctx)
    info = levels[l]
    n, nnz = info["n"], info["nnz"]
    last = l == len(levels) - 1
    rp = np.zeros(n + 1, dtype=np.int32)
    ci = np.zeros(nnz, dtype=np.int32)
    va = np.zeros(nnz, dtype=np.float64)
    agg = None if last else np.zeros(n, dtype=np.int32)
    col = None if last else np.zeros(n, dtype=np.int32)
    _check(lib().amg_export_level(ctx, l, _ptr(rp), _ptr(ci), _ptr(va), _ptr(agg), _ptr(col)),
           "amg_export_level")
    return dict(row_ptr=rp, col=ci, val=va, agg=agg, colour=col, **info)


def _host_csr(row_ptr, col, val):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    A = amg_csr(int(row_ptr.shape[0]) - 1, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val), 0)
    return A, (row_ptr, col, val)


def amg_aggregate(row_ptr, col, val, params: amg_params):
    """Host aggregation of one level; returns (agg, n_coarse)."""
    A, keep = _host_csr(row_ptr, col, val)
    agg = np.zeros(A.n, dtype=np.int32)
    nc = _c_i32()
    _check(lib().amg_aggregate(ctypes.byref(A), ctypes.byref(params), _ptr(agg), ctypes.byref(nc)),
           "amg_aggregate")
    return agg, int(nc.value)


def amg_colour(row_ptr, col, val):
    A, keep = _host_csr(row_ptr, col, val)
    colour = np.zeros(A.n, dtype=np.int32)
    nc = _c_i32()
    _check(lib().amg_colour(ctypes.byref(A), _ptr(colour), ctypes.byref(nc)), "amg_colour")
    return colour, int(nc.value)


def amg_profile_enable(ctx: int, enable) -> None:
    """enable: 0 off, 1 (or True) per kernel, 2 per graph launch."""
    _check(lib().amg_profile_enable(ctx, int(enable)), "amg_profile_enable")


def amg_profile_read(ctx: int) -> list:
    n = _check(lib().amg_profile_read(ctx, None, 0), "amg_profile_read")
    arr = (amg_kernel_stat * max(n, 1))()
    _check(lib().amg_profile_read(ctx, arr, n), "amg_profile_read")
    out = []
    for k in range(n):
        d = struct_dict(arr[k])
        d["name"] = arr[k].name.decode()
        out.append(d)
    return out


def amg_free(ctx: int) -> None:
    if ctx:
        lib().amg_free(ctx)


def amg_last_error() -> str:
    m = lib().amg_last_error()
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# convenience wrapper used by tests and the benchmark
# ---------------------------------------------------------------------------

class AMG:
    """Owns one context.  Matrices from numpy (host) arrays; vectors as torch
    CUDA float64 tensors."""

    def __init__(self, row_ptr, col, val, dim: int = 3, precision: int = AMG_FP64,
                 stream=None, **overrides):
        self.params = amg_params_default(dim)
        for k, v in overrides.items():
            setattr(self.params, k, v)
        self.params.precision = precision
        if stream is not None:
            self.params.cuda_stream = int(stream.cuda_stream)
        self.ctx = amg_setup(row_ptr, col, val, self.params)
        self.n = int(row_ptr.shape[0]) - 1

    def close(self):
        if getattr(self, "ctx", None):
            amg_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: int, flexible_cg: int = -1):
        amg_set_precision(self.ctx, precision, flexible_cg)

    def vcycle(self, r_dev, z_dev=None):
        import torch
        if z_dev is None:
            z_dev = torch.empty_like(r_dev)
        amg_vcycle(self.ctx, r_dev, z_dev)
        return z_dev

    def solve(self, b_dev, x_dev=None, tol: float = 1e-8, maxit: int = 500):
        import torch
        if x_dev is None:
            x_dev = torch.zeros_like(b_dev)
        rc, info = amg_pcg_solve(self.ctx, b_dev, x_dev, tol, maxit)
        return x_dev, rc, struct_dict(info)

    def solve_bicgstab(self, b_dev, x_dev=None, tol: float = 1e-8, maxit: int = 500):
        import torch
        if x_dev is None:
            x_dev = torch.zeros_like(b_dev)
        rc, info = amg_bicgstab_solve(self.ctx, b_dev, x_dev, tol, maxit)
        return x_dev, rc, struct_dict(info)

    def solve_host(self, b_host: np.ndarray, x_host: np.ndarray, tol: float = 1e-8,
                   maxit: int = 500, zero_guess: bool = False):
        """x_host holds x_0 on entry (ignored with zero_guess) and x on exit."""
        f = amg_pcg_solve_host_zero_guess if zero_guess else amg_pcg_solve_host
        rc, info = f(self.ctx, b_host, x_host, tol, maxit)
        return rc, struct_dict(info)

    def residual_norm(self, b_dev, x_dev) -> float:
        return amg_residual_norm(self.ctx, b_dev, x_dev)

    def info(self):
        return amg_hierarchy_info(self.ctx)

    def profile(self, enable):
        amg_profile_enable(self.ctx, enable)

    def profile_read(self) -> list:
        return amg_profile_read(self.ctx)

    def level(self, l: int) -> dict:
        return amg_export_level(self.ctx, l)

    def set_level_shape(self, l: int, lanes_per_row: int, threads_per_block: int = 0) -> None:
        amg_set_level_shape(self.ctx, l, lanes_per_row, threads_per_block)

    def set_level_carveout(self, l: int, percent: int) -> None:
        amg_set_level_carveout(self.ctx, l, percent)


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

def amg_server_params_default(dim: int) -> amg_server_params:
    p = amg_server_params()
    _check(lib().amg_server_params_default(ctypes.byref(p), dim), "amg_server_params_default")
    return p


def amg_server_create(params: amg_server_params) -> int:
    h = _c_vp()
    _check(lib().amg_server_create(ctypes.byref(params), ctypes.byref(h)), "amg_server_create")
    return h.value


def amg_submit(server: int, row_ptr, col, val, b, tol: float) -> int:
    """Host (numpy) matrix and right-hand side; both are copied."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    A = amg_csr(int(row_ptr.shape[0]) - 1, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val), 0)
    t = ctypes.c_uint64()
    _check(lib().amg_submit(server, ctypes.byref(A), _ptr(b), float(tol), ctypes.byref(t)),
           "amg_submit")
    return t.value


def amg_poll(server: int, ticket: int, x_out: Optional[np.ndarray]):
    """Returns (rc, info dict, times dict); rc == AMG_PENDING while unfinished.
    Negative solve statuses (ENOTCONV, ...) are returned, not raised; an
    unknown ticket raises."""
    info = amg_solve_info()
    times = amg_request_times()
    rc = lib().amg_poll(server, ticket, _ptr(x_out), ctypes.byref(info), ctypes.byref(times))
    if rc == AMG_ENOTFOUND:
        _check(rc, "amg_poll")
    return rc, struct_dict(info), struct_dict(times)


def amg_server_stats_read(server: int) -> dict:
    st = amg_server_stats()
    _check(lib().amg_server_stats_read(server, ctypes.byref(st)), "amg_server_stats_read")
    return struct_dict(st)


def amg_server_destroy(server: int) -> None:
    if server:
        lib().amg_server_destroy(server)


class Server:
    """Owns one server.  submit() takes numpy CSR + b and returns a ticket;
    poll() returns None while pending, else (status, x, info, times)."""

    def __init__(self, dim: int = 3, **overrides):
        self.params = amg_server_params_default(dim)
        for k, v in overrides.items():
            if hasattr(self.params.params, k) and k not in ("max_slots", "setup_threads", "maxit",
                                                             "hbm_budget_bytes", "batch_vcycles"):
                setattr(self.params.params, k, v)
            else:
                setattr(self.params, k, v)
        self.handle = amg_server_create(self.params)
        self._n = {}

    def submit(self, row_ptr, col, val, b, tol: float = 1e-8) -> int:
        t = amg_submit(self.handle, row_ptr, col, val, b, tol)
        self._n[t] = int(np.asarray(row_ptr).shape[0]) - 1
        return t

    def poll(self, ticket: int):
        x = np.empty(self._n[ticket])
        rc, info, times = amg_poll(self.handle, ticket, x)
        if rc == AMG_PENDING:
            return None
        del self._n[ticket]
        return rc, x, info, times

    def stats(self) -> dict:
        return amg_server_stats_read(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            amg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
