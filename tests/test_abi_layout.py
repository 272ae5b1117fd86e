"""The ctypes structures of the Python binding against the C header: every
structure's size and every field's offset, as a C compiler lays them out
(include/amg.h compiled with the host compiler), so that a field added on one
side only is caught without a GPU."""

import ctypes
import os
import shutil
import subprocess

import pytest

from conftest import ROOT
from paper_1209_0960_gb300 import amg

STRUCTS = ["amg_csr", "amg_params", "amg_solve_info", "amg_level_info", "amg_summary",
           "amg_kernel_stat", "amg_server_params", "amg_request_times", "amg_server_stats"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "amg.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(amg, s)._fields_:
            lines.append(f'  printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        s, name, v = line.split()
        layout[(s, name)] = int(v)
    return layout


@pytest.mark.parametrize("struct", STRUCTS)
def test_binding_structures_match_the_header(c_layout, struct):
    cls = getattr(amg, struct)
    assert ctypes.sizeof(cls) == c_layout[(struct, "size")], struct
    for name, _ in cls._fields_:
        assert getattr(cls, name).offset == c_layout[(struct, name)], f"{struct}.{name}"


def test_noalloc_binding_refuses_cpu_tensors_and_wrong_dtypes():
    # the Python binding checks device, dtype and contiguity before calling the
    # library, so no CPU tensor reaches a kernel
    torch = pytest.importorskip("torch")
    i32 = torch.zeros(5, dtype=torch.int32)
    f64 = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        amg.amg_residual_norm_noalloc(i32, i32, f64, f64, f64, f64[:1])
    import numpy as np
    with pytest.raises(ValueError, match="CUDA tensor"):
        amg.amg_residual_norm_noalloc(np.zeros(5, np.int32), i32, f64, f64, f64, f64)


def test_noalloc_entry_point_refuses_host_pointers():
    # the library refuses host memory itself (cudaPointerGetAttributes): on a
    # machine without a GPU the query fails, with a GPU the pointers are
    # reported as host memory; AMG_EINVAL either way, and nothing is launched
    import numpy as np
    rp = np.arange(5, dtype=np.int32)
    ci = np.arange(4, dtype=np.int32)
    va = np.ones(4)
    b, x, out = np.ones(4), np.zeros(4), np.zeros(1)
    A = amg.amg_csr(4, 4, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 1)
    rc = amg.lib().amg_residual_norm_noalloc(ctypes.byref(A), b.ctypes.data, x.ctypes.data,
                                             out.ctypes.data, None)
    assert rc == amg.AMG_EINVAL
    assert "A->row_ptr" in amg.amg_last_error()
    assert out[0] == 0.0
