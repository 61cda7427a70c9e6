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


def test_density_workspace_follows_the_layout(lib):
    # host-side size queries against the layout of the workspace: (7 + m)
    # dense FP64 blocks per subgraph on the FP64 path; on the split path a
    # tiled-class scratch (16 + 2m staged images of 128 nrb x npmax FP16 hi
    # and lo parts per CTA) only when a subgraph exceeds 128 orbitals; one
    # response image per RHS and CTA; argument errors before any sizing
    from paper_2212_01997_gb300 import _lib

    def size(max_sub, m, precision, n_sub=100, n=600):
        sub_nnz = n_sub * max_sub
        p = _lib.gb_part(n, n_sub, max_sub, 6, sub_nnz, sub_nnz * 6, sub_nnz, None, None, None, None, None)
        o = _lib.gb_opts(precision, 0, 0.0, 0, 0, 0.0)
        nb = ctypes.c_size_t()
        st = lib.gb_density_workspace_size(ctypes.byref(p), m, ctypes.byref(o), ctypes.byref(nb))
        return st, nb.value

    for m in (0, 1, 6):
        st, fp64 = size(100, m, 0)
        assert st == 0 and fp64 >= (7 + m) * 100 * (100 * 100) * 8
    st, small = size(128, 1, 1)
    st2, big = size(200, 1, 1)
    assert st == 0 and st2 == 0
    npmax, nrb = 208, 2
    assert big - small >= 100 * (16 + 2) * (2 * 128 * nrb * npmax * 2)
    assert size(128, 2, 1)[1] > size(128, 1, 1)[1] > size(128, 0, 1)[1]
    assert size(100, 1, 3)[1] >= 100 * (100 * 100) * 8          # eigenvectors of every subgraph
    assert size(100, 9, 1)[0] == 1 and size(100, -1, 0)[0] == 1  # m beyond 8 RHS, negative m
    assert size(100, 1, 0, n_sub=0)[0] == 1


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2212_01997_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "synth" not in src, f


def test_device_errors_name_their_cause(lib):
    # without a usable GPU, gb_create fails with GB_ERR_DEVICE and the CUDA
    # error behind it is reported (gb_last_device_error), not left at success
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: gb_create succeeds")
    h = ctypes.c_void_p()
    assert lib.gb_create(ctypes.byref(h), None) == 7
    name = ctypes.c_char_p()
    code = lib.gb_last_device_error(ctypes.byref(name))
    assert code != 0 and name.value.startswith(b"cuda") and name.value != b"cudaSuccess"
    from paper_2212_01997_gb300 import _lib
    assert "CUDA error" in str(_lib.GbError("gb_create", 7))


def test_noalloc_scratch_holds_the_largest_accepted_partition(lib):
    # the allocation-free partition runs gb_partition's code in a fixed array:
    # that array must hold gb_partition's workspace at the largest size it
    # accepts (65,536 vertices and groups), for any number of edges
    cap = lib.gb_partition_noalloc_scratch_bytes()
    for nnz in (0, 10 ** 6, 10 ** 9):
        for groups in (0, 1, 65536):
            assert lib.gb_partition_workspace_size(65536, nnz, groups) <= cap
    assert 2_000_000 < cap < 2_200_000        # "about 2.1 MB", as the header states
