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
