"""The Python binding's ctypes structures and constants against the C header, without a GPU: a
small C program compiled against include/grape_hg.h prints sizeof / offsetof of every field the
binding declares and the enum values it mirrors."""

import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2304_06200_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [("grape_op", _abi.GrapeOp), ("grape_desc", _abi.GrapeDesc), ("grape_info", _abi.GrapeInfo),
           ("grape_kernel_times_t", _abi.GrapeKernelTimes), ("grape_batch_info_t", _abi.GrapeBatchInfo)]
ENUMS = ["GRAPE_CSR", "GRAPE_DENSE", "GRAPE_FP64", "GRAPE_FP32_BULK", "GRAPE_TC_FP16", "GRAPE_TC_BF16",
         "GRAPE_PROP_TAYLOR", "GRAPE_PROP_EIG"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "grape_hg.h"', "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("off {cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    for e in ENUMS + sorted(_abi.STATUS.values()):
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr   # a field the binding names that the header lacks fails here
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        kind, key, val = line.split()
        table[(kind, key)] = int(val)
    return table


@pytest.mark.parametrize("cname,cls", STRUCTS)
def test_struct_sizes_and_offsets_match_the_header(c_layout, cname, cls):
    assert C.sizeof(cls) == c_layout[("size", cname)]
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[("off", f"{cname}.{field}")], field


def test_enum_values_match_the_header(c_layout):
    for e in ENUMS:
        assert getattr(_abi, e) == c_layout[("enum", e)], e
    for code, name in _abi.STATUS.items():
        assert c_layout[("enum", name)] == code, name
