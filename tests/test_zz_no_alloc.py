"""gb_partition_noalloc: the partition for callers that cannot allocate.

Some callers cannot allocate device memory -- a host framework that owns a
pre-sized pool, or code that must not allocate while it runs -- so the library
offers this one entry point whose scratch lives in a fixed array compiled into
the library.  This file is collected last on purpose; its test must pass both
alone in a fresh process (the first call looks up the array on the device)
and after every other test.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from synth import make_workload
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2212_01997_gb300 as gb
    from paper_2212_01997_gb300 import build
    build.build()
    return gb


def _noalloc(lib, L, G, groups, n_groups, cap):
    n = G.n
    dev = G.ptr.device
    out = {k: torch.full((n + 1,), -7, dtype=torch.int64, device=dev) for k in ("core_ptr", "sub_ptr")}
    out.update({k: torch.full((n,), -7, dtype=torch.int32, device=dev) for k in ("core_idx", "core_pos")})
    out["sub_idx"] = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    p = L.gb_part(n, 0, 0, 0, 0, 0, cap, out["core_ptr"].data_ptr(), out["core_idx"].data_ptr(),
                  out["core_pos"].data_ptr(), out["sub_ptr"].data_ptr(), out["sub_idx"].data_ptr())
    gs = G.struct()
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    st = lib.gb_partition_noalloc(stream, C.byref(gs), C.c_void_p(groups.data_ptr()), n_groups, 0, C.byref(p))
    return st, p, out


def test_noalloc_partition_matches_gb_partition_twice(gb):
    from paper_2212_01997_gb300 import _lib as L
    lib = L.load()
    assert 0 < lib.gb_partition_noalloc_scratch_bytes() < 4 << 20
    for name in ("water64", "water1k"):
        wl, system, _ = make_workload(name, n_rhs=0)
        G = gb.graph_build(to_device(system.H), wl.tau)
        groups = torch.as_tensor(system.orb_group, device=G.ptr.device)
        n_groups = int(system.orb_group.max()) + 1
        ref = gb.partition(G, groups, n_groups)
        for call in range(2):  # two calls in a row share the scratch array
            st, p, out = _noalloc(lib, L, G, groups, n_groups, ref.sub_nnz + 5)
            assert st == 0, L.STATUS.get(st, st)
            assert (p.n_sub, p.max_sub, p.max_core, p.sub_nnz, p.out_nnz) == \
                (ref.n_sub, ref.max_sub, ref.max_core, ref.sub_nnz, ref.out_nnz)
            k = ref.n_sub + 1
            assert torch.equal(out["core_ptr"][:k], ref.core_ptr)
            assert torch.equal(out["sub_ptr"][:k], ref.sub_ptr)
            assert torch.equal(out["core_idx"], ref.core_idx)
            assert torch.equal(out["core_pos"], ref.core_pos)
            assert torch.equal(out["sub_idx"][: ref.sub_nnz], ref.sub_idx)


def test_noalloc_rejects_sizes_beyond_its_scratch(gb):
    from paper_2212_01997_gb300 import _lib as L
    lib = L.load()
    n = 65537  # one above GB_NOALLOC_MAX_VERTICES
    dev = torch.device("cuda")
    ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    idx = torch.zeros(1, dtype=torch.int32, device=dev)
    g = L.gb_graph(n, 0, 0, ptr.data_ptr(), idx.data_ptr())
    bufs = [torch.zeros(n + 1, dtype=torch.int64, device=dev) for _ in range(2)] + \
        [torch.zeros(n, dtype=torch.int32, device=dev) for _ in range(3)]
    p = L.gb_part(n, 0, 0, 0, 0, 0, n, bufs[0].data_ptr(), bufs[2].data_ptr(), bufs[3].data_ptr(),
                  bufs[1].data_ptr(), bufs[4].data_ptr())
    st = lib.gb_partition_noalloc(None, C.byref(g), None, 0, 6, C.byref(p))
    assert st == 3  # GB_ERR_WORKSPACE, nothing launched
    assert torch.all(bufs[0] == 0)
