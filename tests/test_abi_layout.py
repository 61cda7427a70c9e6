"""The Python binding's view of the C ABI matches include/gbqr.h (CPU only).

The binding declares every struct of the header as a ctypes Structure and
every entry point's argument list.  A drift between the two would pass
garbage through the boundary without any error, so this checks them against
the header itself: a small C program, compiled with the host compiler,
prints the size of each struct and the offset of each field, and every
prototype's parameter count is read from the header text.
"""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2212_01997_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbqr.h")
STRUCTS = [_lib.gb_csr, _lib.gb_csc, _lib.gb_graph, _lib.gb_part, _lib.gb_opts, _lib.gb_report, _lib.gb_plan,
           _lib.gb_blocks]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gbqr.h"', "int main(void) {"]
    for s in STRUCTS:
        name = s.__name__
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in s._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for s in STRUCTS:
        name = s.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(s), name
        for field, _ in s._fields_:
            assert got[(name, field)] == getattr(s, field).offset, (name, field)


def _prototypes():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"^\s*(?:int|int64_t|size_t|const char\*)\s+(gb_\w+)\s*\(([^)]*)\)\s*;", text,
                         flags=re.M | re.S):
        params = m.group(2).strip()
        protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return protos


def test_entry_point_arities_match_the_header():
    protos = _prototypes()
    assert len(protos) == len(_lib.SIGNATURES)
    for name, _, args in _lib.SIGNATURES:
        assert protos[name] == len(args), name


def test_status_and_precision_codes_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    names = list(_lib.STATUS.values()) + ["GB_PREC_FP64", "GB_PREC_FP16X3", "GB_PREC_BF16X3", "GB_PREC_EIGEN"]
    src = tmp_path / "codes.c"
    src.write_text("\n".join(['#include <stdio.h>', '#include "gbqr.h"', "int main(void) {"] +
                             [f'printf("{n} %d\\n", (int){n});' for n in names] + ["return 0;", "}"]))
    exe = tmp_path / "codes"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {line.split()[0]: int(line.split()[1]) for line in out if line}
    assert {v: k for k, v in _lib.STATUS.items()} == {n: got[n] for n in _lib.STATUS.values()}
    prec = {"fp64": "GB_PREC_FP64", "fp16x3": "GB_PREC_FP16X3", "bf16x3": "GB_PREC_BF16X3", "eigen": "GB_PREC_EIGEN"}
    assert {k: got[v] for k, v in prec.items()} == _lib.PRECISION
