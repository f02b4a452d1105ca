"""The binding's ctypes structures have the C layout of include/fdas.h:
a small C program (compiled here with the host compiler) prints offsetof
and sizeof of every field, and each must equal the ctypes field offset."""
import ctypes
import json
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = ["fdas_opts", "fdas_series", "fdas_candidate", "fdas_plan_info", "fdas_seed",
           "fdas_refined", "fdas_profile", "fdas_dedisp_info"]


@pytest.fixture(scope="module")
def capi():
    from paper_2211_13517_gb300 import capi as c
    return c


def test_struct_offsets_match_the_header(capi):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fdas.h"', "int main(void) {",
             '  printf("{");']
    first = True
    for sname in STRUCTS:
        st = getattr(capi, sname)
        fields = [f[0] for f in st._fields_]
        sep = "" if first else ","
        first = False
        lines.append(f'  printf("{sep}\\"{sname}\\": {{\\"size\\": %zu", sizeof({sname}));')
        for f in fields:
            lines.append(f'  printf(", \\"{f}\\": %zu", offsetof({sname}, {f}));')
        lines.append('  printf("}");')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    for sname in STRUCTS:
        st = getattr(capi, sname)
        assert out[sname]["size"] == ctypes.sizeof(st), sname
        for f in st._fields_:
            assert out[sname][f[0]] == getattr(st, f[0]).offset, (sname, f[0])
