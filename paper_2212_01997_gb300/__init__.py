"""GB300-native graph-based density matrix and canonical response.

Thin Python binding over the C ABI of ``libgbqr.so`` (include/gbqr.h): the
functions below only marshal torch device tensors into the C structs and grow
caller-owned workspaces; every step of the computation runs in the CUDA
kernels of the library.  PyTorch provides device memory and the stream.

    G = graph_build(H, tau, paths2=False, d_prev=None)
    P = partition(G, groups=orbital_molecule_ids, n_groups=n_molecules)
    R = density_and_response(H, [H1], kT, n_electrons, P, precision="fp16x3")
    R.D, R.D1[0], R.mu, R.mu1[0]
"""

from __future__ import annotations

import ctypes as C
import math
from ctypes import byref as C_byref, c_double as C_double, c_int32 as C_int32
from dataclasses import dataclass, field

import torch

from . import _lib as L
from ._lib import GbError, PRECISION

__all__ = ["DeviceCSR", "Graph", "Partition", "CSC", "Result", "Handle", "graph_build", "partition",
           "density_and_response", "mulliken_charges", "preconditioner", "krylov_update", "plan_autotune",
           "GbError", "PRECISION", "library"]


def library():
    """The loaded libgbqr.so (raises if it has not been built)."""
    return L.load()


def Cn(coupling: "DeviceCSR") -> int:
    """Rows of a coupling matrix (atoms)."""
    return int(coupling.n)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


@dataclass
class DeviceCSR:
    """Square CSR matrix on the GPU: ptr int64 (n+1), idx int32, val float64."""

    n: int
    ptr: torch.Tensor
    idx: torch.Tensor
    val: torch.Tensor

    @staticmethod
    def from_arrays(n, indptr, indices, data, device="cuda") -> "DeviceCSR":
        return DeviceCSR(int(n), torch.as_tensor(indptr, dtype=torch.int64).to(device),
                         torch.as_tensor(indices, dtype=torch.int32).to(device),
                         torch.as_tensor(data, dtype=torch.float64).to(device))

    @property
    def nnz(self) -> int:
        return int(self.idx.numel())

    def struct(self) -> L.gb_csr:
        return L.gb_csr(self.n, self.nnz, _ptr(self.ptr), _ptr(self.idx), _ptr(self.val))


@dataclass
class Graph:
    n: int
    ptr: torch.Tensor
    idx: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.idx.numel())

    def struct(self) -> L.gb_graph:
        return L.gb_graph(self.n, self.nnz, self.nnz, _ptr(self.ptr), _ptr(self.idx))


@dataclass
class Partition:
    n: int
    n_sub: int
    max_sub: int
    max_core: int
    sub_nnz: int
    out_nnz: int
    core_ptr: torch.Tensor
    core_idx: torch.Tensor
    core_pos: torch.Tensor
    sub_ptr: torch.Tensor
    sub_idx: torch.Tensor

    def struct(self) -> L.gb_part:
        return L.gb_part(self.n, self.n_sub, self.max_sub, self.max_core, self.sub_nnz, self.out_nnz,
                         self.sub_idx.numel(), _ptr(self.core_ptr), _ptr(self.core_idx),
                         _ptr(self.core_pos), _ptr(self.sub_ptr), _ptr(self.sub_idx))


@dataclass
class CSC:
    """Collected ragged CSC matrix: column j holds rows S_i of its subgraph."""

    n: int
    ptr: torch.Tensor
    idx: torch.Tensor
    val: torch.Tensor

    def struct(self, with_index=True) -> L.gb_csc:
        return L.gb_csc(self.n, self.val.numel(), self.val.numel(),
                        _ptr(self.ptr) if with_index else None,
                        _ptr(self.idx) if with_index else None, _ptr(self.val))


@dataclass
class Result:
    mu: float
    mu1: list
    D: CSC
    D1: list
    status: int
    report: dict = field(default_factory=dict)


class Handle:
    """A gb_handle bound to one CUDA stream, with a growable workspace."""

    def __init__(self, stream: torch.cuda.Stream | None = None, device=None):
        self.lib = L.load()
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check("gb_create", self.lib.gb_create(C.byref(h), C.c_void_p(self.stream.cuda_stream)))
        self.h = h
        self.ws = None

    def workspace(self, nbytes: int) -> None:
        nbytes = max(int(nbytes), 256)
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = torch.empty(int(nbytes * 1.05) + 4096, dtype=torch.uint8, device=self.device)
        L.check("gb_set_workspace", self.lib.gb_set_workspace(self.h, self.ws.data_ptr(), self.ws.numel()))

    def __del__(self):
        try:
            if getattr(self, "h", None) and self.h.value:
                self.lib.gb_destroy(self.h)
        except Exception:
            pass


_handles: dict = {}


def _default_handle(device=None) -> Handle:
    dev = torch.device(device or "cuda")
    stream = torch.cuda.current_stream(dev)
    key = (dev.index, stream.cuda_stream)
    if key not in _handles:
        _handles[key] = Handle(stream, dev)
    return _handles[key]


def graph_build(H: DeviceCSR, tau: float, *, paths2: bool = False, d_prev: CSC | None = None,
                handle: Handle | None = None) -> Graph:
    """gb_graph_build: thresholded, symmetrised graph (+ paths of length two)."""
    hd = handle or _default_handle(H.ptr.device)
    lib = hd.lib
    nnz_d = 0 if d_prev is None else d_prev.val.numel()
    hd.workspace(lib.gb_graph_build_workspace_size(H.n, H.nnz, nnz_d, int(paths2)))
    cap = max(1, 2 * (H.nnz + nnz_d) * (8 if paths2 else 1))
    hs = H.struct()
    ds = None if d_prev is None else C.byref(d_prev.struct())
    for _ in range(3):
        ptr = torch.empty(H.n + 1, dtype=torch.int64, device=hd.device)
        idx = torch.empty(cap, dtype=torch.int32, device=hd.device)
        g = L.gb_graph(H.n, 0, cap, ptr.data_ptr(), idx.data_ptr())
        st = lib.gb_graph_build(hd.h, C.byref(hs), ds, float(tau), int(paths2), C.byref(g))
        if st == 2:  # GB_ERR_CAPACITY
            cap = int(g.nnz) + 1
            continue
        L.check("gb_graph_build", st)
        return Graph(H.n, ptr, idx[: g.nnz])
    raise GbError("gb_graph_build", 2)


def partition(G: Graph, groups: torch.Tensor | None = None, n_groups: int | None = None, *,
              target_core_size: int = 6, subgroups: torch.Tensor | None = None,
              n_subgroups: int | None = None, max_sub: int = 0, handle: Handle | None = None) -> Partition:
    """gb_partition: disjoint cores (one per group id, or blocks) and distance-1 halos.

    With ``subgroups`` and ``max_sub`` (gb_partition_capped), cores whose
    subgraph exceeds ``max_sub`` are replaced by their subgroups.
    """
    hd = handle or _default_handle(G.ptr.device)
    lib = hd.lib
    n = G.n
    dev = hd.device
    if groups is not None:
        groups = groups.to(device=dev, dtype=torch.int32).contiguous()
        if n_groups is None:
            n_groups = int(groups.max().item()) + 1
    capped = subgroups is not None and max_sub > 0
    if capped:
        if groups is None:
            raise ValueError("a capped partition needs group ids")
        subgroups = subgroups.to(device=dev, dtype=torch.int32).contiguous()
        if n_subgroups is None:
            n_subgroups = int(subgroups.max().item()) + 1
        hd.workspace(lib.gb_partition_capped_workspace_size(n, G.nnz, int(n_groups), int(n_subgroups)))
    else:
        hd.workspace(lib.gb_partition_workspace_size(n, G.nnz, int(n_groups or 0) if groups is not None else 0))
    core_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    core_idx = torch.empty(n, dtype=torch.int32, device=dev)
    core_pos = torch.empty(n, dtype=torch.int32, device=dev)
    sub_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    cap = max(1, G.nnz + n)
    gs = G.struct()
    for _ in range(3):
        sub_idx = torch.empty(cap, dtype=torch.int32, device=dev)
        p = L.gb_part(n, 0, 0, 0, 0, 0, cap, core_ptr.data_ptr(), core_idx.data_ptr(),
                      core_pos.data_ptr(), sub_ptr.data_ptr(), sub_idx.data_ptr())
        if capped:
            st = lib.gb_partition_capped(hd.h, C.byref(gs), groups.data_ptr(), int(n_groups), subgroups.data_ptr(),
                                         int(n_subgroups), int(max_sub), C.byref(p))
        else:
            st = lib.gb_partition(hd.h, C.byref(gs), None if groups is None else groups.data_ptr(),
                                  int(n_groups or 0), int(target_core_size), C.byref(p))
        if st == 2:
            cap = int(p.sub_nnz) + 1
            continue
        L.check("gb_partition_capped" if capped else "gb_partition", st)
        return Partition(n, p.n_sub, p.max_sub, p.max_core, p.sub_nnz, p.out_nnz,
                         core_ptr[: p.n_sub + 1], core_idx, core_pos, sub_ptr[: p.n_sub + 1],
                         sub_idx[: p.sub_nnz])
    raise GbError("gb_partition", 2)


def density_and_response(H: DeviceCSR, H1: list, kT: float, n_electrons: float, part: Partition, *,
                         precision: str = "fp64", mu0: float = math.nan, max_newton: int = 0,
                         tol_occ: float = 0.0, min_steps: int = 0, ns_iters: int = 0, tol_d: float = 0.0,
                         split_small_npad: int = 0, refine_d1: float = 0.0, out: tuple | None = None,
                         handle: Handle | None = None, raise_on_error: bool = True) -> Result:
    """gb_density_and_response: D, D1, mu, mu1 on the partitioned graph.

    ``out`` may pass preallocated (D, [D1...]) CSC containers to reuse.
    """
    hd = handle or _default_handle(H.ptr.device)
    lib = hd.lib
    m = len(H1)
    opts = L.gb_opts(PRECISION[precision], int(max_newton), float(tol_occ), int(min_steps), int(ns_iters),
                     float(tol_d), int(split_small_npad), float(refine_d1))
    ps = part.struct()
    nbytes = C.c_size_t()
    L.check("gb_density_workspace_size", lib.gb_density_workspace_size(C.byref(ps), m, C.byref(opts),
                                                                         C.byref(nbytes)))
    hd.workspace(nbytes.value)
    dev = hd.device
    if out is None:
        D = CSC(part.n, torch.empty(part.n + 1, dtype=torch.int64, device=dev),
                torch.empty(part.out_nnz, dtype=torch.int32, device=dev),
                torch.empty(part.out_nnz, dtype=torch.float64, device=dev))
        D1 = [CSC(part.n, D.ptr, D.idx, torch.empty(part.out_nnz, dtype=torch.float64, device=dev))
              for _ in range(m)]
    else:
        D, D1 = out
    hs = H.struct()
    h1s = (L.gb_csr * max(m, 1))(*[h.struct() for h in H1])
    ds = D.struct()
    d1s = (L.gb_csc * max(m, 1))(*[d.struct(with_index=False) for d in D1])
    mu = C.c_double(mu0)
    mu1 = (C.c_double * max(m, 1))()
    rep = L.gb_report()
    st = lib.gb_density_and_response(hd.h, C.byref(hs), h1s, m, float(kT), float(n_electrons),
                                     C.byref(ps), C.byref(opts), C.byref(mu), C.byref(ds), d1s, mu1,
                                     C.byref(rep))
    if raise_on_error:
        L.check("gb_density_and_response", st)
    report = {k: getattr(rep, k) for k, _ in L.gb_report._fields_}
    return Result(mu.value, [mu1[r] for r in range(m)], D, D1, st, report)


def mulliken_charges(D: CSC, D1: list, atom_ptr: torch.Tensor, atom_orb: torch.Tensor, z_val: torch.Tensor, *,
                     handle: Handle | None = None) -> tuple:
    """gb_mulliken_charges: q_I = Z_I - 2 sum_o D_oo and q1_r,I = -2 sum_o D1_r,oo.

    ``atom_ptr`` / ``atom_orb``: the orbitals of each atom (CSR); ``z_val``:
    valence charges.  Returns (q, [q1_r ...]) as device tensors.
    """
    hd = handle or _default_handle(D.val.device)
    lib = hd.lib
    dev = hd.device
    m = len(D1)
    atom_ptr = atom_ptr.to(device=dev, dtype=torch.int64).contiguous()
    atom_orb = atom_orb.to(device=dev, dtype=torch.int32).contiguous()
    z_val = z_val.to(device=dev, dtype=torch.float64).contiguous()
    n_atoms = atom_ptr.numel() - 1
    hd.workspace(lib.gb_mulliken_workspace_size())
    q = torch.empty(n_atoms, dtype=torch.float64, device=dev)
    q1 = torch.empty((max(m, 1), n_atoms), dtype=torch.float64, device=dev)
    ds = D.struct()
    d1s = (L.gb_csc * max(m, 1))(*[d.struct(with_index=False) for d in D1])
    L.check("gb_mulliken_charges", lib.gb_mulliken_charges(hd.h, C.byref(ds), d1s, m, n_atoms, atom_ptr.data_ptr(),
                                                             atom_orb.data_ptr(), z_val.data_ptr(), q.data_ptr(),
                                                             q1.data_ptr() if m else None))
    return q, [q1[r] for r in range(m)]


@dataclass
class Blocks:
    """Block-diagonal preconditioner K0: block k over atoms[atom_ptr[k]:atom_ptr[k+1]], row-major at
    val[val_ptr[k]:]."""

    atom_ptr: torch.Tensor
    atoms: torch.Tensor
    val_ptr: torch.Tensor
    val: torch.Tensor
    mu: float

    def struct(self) -> L.gb_blocks:
        return L.gb_blocks(self.atom_ptr.numel() - 1, self.atoms.numel(), self.val.numel(), self.val.numel(),
                           self.atom_ptr.data_ptr(), self.atoms.data_ptr(), self.val_ptr.data_ptr(),
                           self.val.data_ptr())


def preconditioner(H: DeviceCSR, part: Partition, kT: float, n_electrons: float, C: DeviceCSR,
                   orb_atom: torch.Tensor, alpha: float, *, mu0: float = math.nan,
                   handle: Handle | None = None) -> Blocks:
    """gb_preconditioner: the subgraph preconditioner k0 = (j_c - alpha I)^-1 per core."""
    hd = handle or _default_handle(H.ptr.device)
    lib = hd.lib
    dev = hd.device
    ps = part.struct()
    hd.workspace(lib.gb_preconditioner_workspace_size(C_byref(ps)))
    orb_atom = orb_atom.to(device=dev, dtype=torch.int32).contiguous()
    atom_ptr = torch.empty(part.n_sub + 1, dtype=torch.int64, device=dev)
    atoms = torch.empty(Cn(C), dtype=torch.int32, device=dev)
    val_ptr = torch.empty(part.n_sub + 1, dtype=torch.int64, device=dev)
    cap = 16 * Cn(C)
    for _ in range(3):
        val = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
        bl = L.gb_blocks(0, 0, 0, val.numel(), atom_ptr.data_ptr(), atoms.data_ptr(), val_ptr.data_ptr(),
                         val.data_ptr())
        hs, cs = H.struct(), C.struct()
        muc = C_double(mu0)
        st = lib.gb_preconditioner(hd.h, C_byref(hs), C_byref(ps), float(kT), float(n_electrons), C_byref(cs),
                                   orb_atom.data_ptr(), Cn(C), float(alpha), C_byref(muc), C_byref(bl))
        if st == 2:
            cap = int(bl.val_nnz)
            continue
        L.check("gb_preconditioner", st)
        return Blocks(atom_ptr, atoms, val_ptr, val[: bl.val_nnz], muc.value)
    raise GbError("gb_preconditioner", 2)


def krylov_update(H0: DeviceCSR, part: Partition, kT: float, n_electrons: float, C: DeviceCSR,
                  orb_atom: torch.Tensor, atom_ptr: torch.Tensor, atom_orb: torch.Tensor, z: torch.Tensor,
                  n: torch.Tensor, m: int, *, K0: Blocks | None = None, k0_scalar: float = -0.5,
                  breakdown: float = 1e-6, precision: str = "fp64", mu0: float = math.nan,
                  handle: Handle | None = None) -> dict:
    """gb_krylov_update: the preconditioned low-rank Krylov update of the populations n."""
    hd = handle or _default_handle(H0.ptr.device)
    lib = hd.lib
    dev = hd.device
    na = Cn(C)
    ps, hs, cs = part.struct(), H0.struct(), C.struct()
    opts = L.gb_opts(PRECISION[precision], 0, 0.0, 0, 0, 0.0, 0)
    hd.workspace(lib.gb_krylov_workspace_size(C_byref(hs), C_byref(ps), na, C_byref(opts)))
    f = torch.empty(na, dtype=torch.float64, device=dev)
    dn = torch.empty(na, dtype=torch.float64, device=dev)
    v = torch.zeros((m, na), dtype=torch.float64, device=dev)
    fv = torch.zeros((m, na), dtype=torch.float64, device=dev)
    Mh = (C_double * (m * m))()
    rank = C_int32(0)
    muc = C_double(mu0)
    conv = [t.to(device=dev).contiguous() for t in (orb_atom.to(torch.int32), atom_ptr.to(torch.int64),
                                                    atom_orb.to(torch.int32), z.to(torch.float64),
                                                    n.to(torch.float64))]
    ks = K0.struct() if K0 is not None else None
    L.check("gb_krylov_update", lib.gb_krylov_update(hd.h, C_byref(hs), C_byref(ps), float(kT), float(n_electrons),
                                                     C_byref(cs), conv[0].data_ptr(), conv[1].data_ptr(),
                                                     conv[2].data_ptr(), na, conv[3].data_ptr(), conv[4].data_ptr(),
                                                     C_byref(ks) if ks is not None else None, float(k0_scalar), int(m),
                                                     float(breakdown), C_byref(opts), C_byref(muc), f.data_ptr(),
                                                     v.data_ptr(), fv.data_ptr(), dn.data_ptr(), Mh,
                                                     C_byref(rank)))
    r = rank.value
    M = [[Mh[i * m + j] for j in range(r)] for i in range(r)]
    return {"f": f, "v": v[:r], "fv": fv[:r], "dn": dn, "M": M, "rank": r, "mu": muc.value}


def plan_autotune(H: DeviceCSR, H1: list, kT: float, n_electrons: float, part: Partition, mu: float, *,
                  precision: str = "fp16x3", min_steps: int = 0, ns_iters: int = 0,
                  out: tuple | None = None, handle: Handle | None = None) -> dict:
    """gb_plan_autotune: the split configuration's size threshold for this partition.

    Times one recursion pass per candidate (at the fixed ``mu``) and returns
    the plan as a dict; pass ``plan["split_small_npad"]`` to
    density_and_response.  The handle caches the plan by the partition's size.
    """
    if precision == "fp64":
        raise ValueError("plan_autotune: the plan is for the split-precision recursion")
    hd = handle or _default_handle(H.ptr.device)
    lib = hd.lib
    m = len(H1)
    opts = L.gb_opts(PRECISION[precision], 1, 0.0, int(min_steps), int(ns_iters), 0.0, 0)
    ps = part.struct()
    nbytes = C.c_size_t()
    L.check("gb_density_workspace_size", lib.gb_density_workspace_size(C.byref(ps), m, C.byref(opts),
                                                                         C.byref(nbytes)))
    hd.workspace(nbytes.value)
    dev = hd.device
    if out is None:
        D = CSC(part.n, torch.empty(part.n + 1, dtype=torch.int64, device=dev),
                torch.empty(part.out_nnz, dtype=torch.int32, device=dev),
                torch.empty(part.out_nnz, dtype=torch.float64, device=dev))
        D1 = [CSC(part.n, D.ptr, D.idx, torch.empty(part.out_nnz, dtype=torch.float64, device=dev))
              for _ in range(m)]
    else:
        D, D1 = out
    hs = H.struct()
    h1s = (L.gb_csr * max(m, 1))(*[h.struct() for h in H1])
    ds = D.struct()
    d1s = (L.gb_csc * max(m, 1))(*[d.struct(with_index=False) for d in D1])
    plan = L.gb_plan()
    L.check("gb_plan_autotune", lib.gb_plan_autotune(hd.h, C.byref(hs), h1s, m, float(kT), float(n_electrons),
                                                       C.byref(ps), C.byref(opts), float(mu), C.byref(ds), d1s,
                                                       C.byref(plan)))
    k = plan.n_candidates
    return {"split_small_npad": plan.split_small_npad, "candidates": list(plan.candidate[:k]),
            "pass_ms": list(plan.pass_ms[:k]), "bin_count": list(plan.bin_count), "cached": bool(plan.cached)}
