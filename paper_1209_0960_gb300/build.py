"""Build libamg.so in-tree for sm_103a (nvcc for the CUDA sources, g++ for the
host-only setup code), compiling translation units in parallel; with
checked=True the same sources with AMG_DEVICE_CHECKS (every solve kernel
tests the indices it gathers) into libamg_checked.so."""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libamg.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libamg_checked.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels.cu", "setup_device.cu", "solver.cu", "noalloc.cu", "server.cu",
              "aggregate_device.cu"]
CPP_SOURCES = ["host_setup.cpp"]
HEADERS = ["device.h", "host_setup.h"]


def _deps():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "amg.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, extra_nvcc=None, checked: bool = False) -> str:
    """Compile libamg.so (libamg_checked.so with checked) if any source is newer
    than it; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    if not os.path.exists(NVCC) and shutil.which("nvcc") is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libamg")
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    tag = ".checked" if checked else ""
    defs = ["-DAMG_DEVICE_CHECKS"] if checked else []
    jobs = []
    objs = []
    for f in CU_SOURCES:
        obj = os.path.join(OUT_DIR, f + tag + ".o")
        objs.append(obj)
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", *defs, *(extra_nvcc or []), *inc,
                     "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, f + tag + ".o")
        objs.append(obj)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *inc,
                     "-I" + os.path.join(CUDA_HOME, "include"), "-c", os.path.join(CSRC, f),
                     "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    tmp = lib + f".tmp{os.getpid()}"
    logs.append(_run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]))
    os.replace(tmp, lib)
    if verbose:
        sys.stdout.write("".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_nvcc=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                checked="--checked" in sys.argv))
