"""The binding's ctypes structures match the C declarations of include/ats.h
field by field: a small C program (gcc, no CUDA) prints sizeof and offsetof
of every ABI struct, and each must equal the ctypes size and field offset
(a reordered, retyped or missing field in either side fails here)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["ats_level_desc", "ats_coef_desc", "ats_solve_opts", "ats_solve_stats", "ats_kernel_stats",
           "ats_tune_result", "ats_hierarchy_desc", "ats_server_opts", "ats_request", "ats_result",
           "ats_server_counters"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    from paper_1401_1112_gb300 import ats

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ats.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(ats, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        name, field, value = line.split()
        table[(name, field)] = int(value)
    return ats, table


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_matches_header(c_layout, name):
    ats, table = c_layout
    cls = getattr(ats, name)
    assert ctypes.sizeof(cls) == table[(name, "size")], name
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == table[(name, field)], (name, field)
