"""The Python binding's view of the C ABI (include/mf.h) matches the header.

paper_2007_00202_gb300/mf.py mirrors the header's structs with ctypes and repeats its constants.
A small C program compiled against the header (gcc, no GPU) prints every struct's size and every
field's offset, and every constant; they must equal what the binding declares, so that an edit
of one side without the other fails here instead of corrupting arguments at run time.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_2007_00202_gb300.mf as mf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [mf.mf_options, mf.mf_solve_info, mf.mf_stats_t, mf.mf_kernel_profile_t, mf.mf_request_info,
           mf.mf_analysis_sizes_t]
CONSTANTS = ["MF_OK", "MF_LATTICE_NODE", "MF_LATTICE_EDGE", "MF_PREC_C64", "MF_PREC_C128", "MF_REFINE_NONE",
             "MF_REFINE_GMRES", "MF_REFINE_IR", "MF_PROF_NARROW_GEMM", "MF_PROF_FRONT_GEMM", "MF_OP_F11",
             "MF_OP_F11_INV", "MF_OP_F12", "MF_OP_F21", "MF_OP_C", "MF_OPTIONS_V1", "MF_OPTIONS_V2",
             "MF_ORDER_AUTO", "MF_ORDER_HYBRID", "MF_ORDER_GRAPH"]


@pytest.fixture(scope="module")
def header_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mf.h"', "int main(void) {"]
    for S in STRUCTS:
        n = S.__name__
        lines.append(f'  printf("size {n} %zu\\n", sizeof({n}));')
        for fname, _ in S._fields_:
            lines.append(f'  printf("off {n} {fname} %zu\\n", offsetof({n}, {fname}));')
    for c in CONSTANTS:
        lines.append(f'  printf("const {c} %ld\\n", (long)({c}));')
    for code, name in mf.ERRORS.items():
        lines.append(f'  printf("const {name} %ld\\n", (long)({name}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        parts = ln.split()
        got[tuple(parts[:-1])] = int(parts[-1])
    return got


@pytest.mark.parametrize("S", STRUCTS, ids=lambda S: S.__name__)
def test_struct_layout_matches_header(header_layout, S):
    import ctypes
    n = S.__name__
    assert header_layout[("size", n)] == ctypes.sizeof(S)
    for fname, _ in S._fields_:
        assert header_layout[("off", n, fname)] == getattr(S, fname).offset, fname


def test_constants_match_header(header_layout):
    for c in CONSTANTS:
        assert header_layout[("const", c)] == getattr(mf, c), c
    for code, name in mf.ERRORS.items():
        assert header_layout[("const", name)] == code, name
