"""The C-ABI library loads and exports every entry point include/gbqr.h declares.

CPU only: the library is cross-compiled here for sm_103a; only host-side
functions (status strings, version, workspace-size queries) are called.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "gbqr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|int64_t|size_t|const char\*)\s+(gb_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_01997_gb300 import build as b
    b.build()
    from paper_2212_01997_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("gb_graph_build", "gb_partition", "gb_density_and_response", "gb_create",
                     "gb_destroy", "gb_set_workspace"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    from paper_2212_01997_gb300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == names


def test_host_side_queries(lib):
    assert lib.gb_status_string(0) == b"GB_OK"
    assert lib.gb_status_string(5) == b"GB_ERR_NO_CONVERGE"
    maj, mnr, arch = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    assert lib.gb_version(ctypes.byref(maj), ctypes.byref(mnr), ctypes.byref(arch)) == 0
    assert arch.value == 103
    a = lib.gb_graph_build_workspace_size(1000, 50000, 0, 0)
    b = lib.gb_graph_build_workspace_size(1000, 50000, 0, 1)
    assert 0 < a < b
    assert lib.gb_partition_workspace_size(1000, 50000, 0) > 0
    # argument errors are reported, not crashed on (no device needed)
    assert lib.gb_graph_build(None, None, None, 0.0, 0, None) == 1
    assert lib.gb_create(None, None) == 1


def test_density_workspace_query(lib):
    from paper_2212_01997_gb300 import _lib
    p = _lib.gb_part(600, 100, 80, 6, 7000, 42000, 7000, None, None, None, None, None)
    o = _lib.gb_opts(0, 0, 0.0, 0, 0, 0.0)
    nb = ctypes.c_size_t()
    assert lib.gb_density_workspace_size(ctypes.byref(p), 1, ctypes.byref(o), ctypes.byref(nb)) == 0
    fp64 = nb.value
    o.precision = 1
    assert lib.gb_density_workspace_size(ctypes.byref(p), 1, ctypes.byref(o), ctypes.byref(nb)) == 0
    assert fp64 > 0 and nb.value > 0
    assert lib.gb_density_workspace_size(ctypes.byref(p), 99, ctypes.byref(o), ctypes.byref(nb)) == 1


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2212_01997_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "synth" not in src, f
