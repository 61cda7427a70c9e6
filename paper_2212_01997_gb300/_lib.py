"""ctypes declarations of the gbqr C ABI (include/gbqr.h).

Loading fails loudly when libgbqr.so is missing: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgbqr.so")

GB_OK = 0
STATUS = {0: "GB_OK", 1: "GB_ERR_ARG", 2: "GB_ERR_CAPACITY", 3: "GB_ERR_WORKSPACE",
          4: "GB_ERR_MU_BRACKET", 5: "GB_ERR_NO_CONVERGE", 6: "GB_ERR_NAN", 7: "GB_ERR_DEVICE",
          8: "GB_ERR_UNSUPPORTED", 9: "GB_ERR_TIMEOUT"}
PRECISION = {"fp64": 0, "fp16x3": 1, "bf16x3": 2, "eigen": 3}


class GbError(RuntimeError):
    def __init__(self, func: str, status: int):
        msg = f"{func} returned {STATUS.get(status, status)}"
        if STATUS.get(status) == "GB_ERR_DEVICE" and _lib is not None:
            name = C.c_char_p()
            code = _lib.gb_last_device_error(C.byref(name))
            msg += f" (CUDA error {code}: {name.value.decode() if name.value else '?'})"
        super().__init__(msg)
        self.status = status


class gb_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("ptr", C.c_void_p), ("idx", C.c_void_p),
                ("val", C.c_void_p)]


class gb_csc(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("capacity", C.c_int64), ("ptr", C.c_void_p),
                ("idx", C.c_void_p), ("val", C.c_void_p)]


class gb_graph(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("capacity", C.c_int64), ("ptr", C.c_void_p),
                ("idx", C.c_void_p)]


class gb_part(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_sub", C.c_int32), ("max_sub", C.c_int32), ("max_core", C.c_int32),
                ("sub_nnz", C.c_int64), ("out_nnz", C.c_int64), ("sub_capacity", C.c_int64),
                ("core_ptr", C.c_void_p), ("core_idx", C.c_void_p), ("core_pos", C.c_void_p),
                ("sub_ptr", C.c_void_p), ("sub_idx", C.c_void_p)]


class gb_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_newton", C.c_int32), ("tol_occ", C.c_double),
                ("min_steps", C.c_int32), ("ns_iters", C.c_int32), ("tol_d", C.c_double),
                ("split_small_npad", C.c_int32), ("refine_d1", C.c_double)]


class gb_report(C.Structure):
    _fields_ = [("passes", C.c_int32), ("max_steps", C.c_int32), ("n_sub", C.c_int32),
                ("max_sub", C.c_int32), ("mu", C.c_double), ("trace_d", C.c_double),
                ("dndmu", C.c_double), ("occ_residual", C.c_double), ("trace_d1mu", C.c_double),
                ("eps_min", C.c_double), ("eps_max", C.c_double), ("gemm_flops", C.c_double),
                ("gemm_flops_per_step_count", C.c_double),
                ("pass_kernel_ms", C.c_double), ("mu_d_bound", C.c_double),
                ("kernel_launches", C.c_int64), ("refined", C.c_int32), ("refine_skipped", C.c_int32),
                ("refine_ms", C.c_double)]


class gb_plan(C.Structure):
    _fields_ = [("split_small_npad", C.c_int32), ("n_candidates", C.c_int32), ("candidate", C.c_int32 * 5),
                ("pass_ms", C.c_double * 5), ("bin_count", C.c_int64 * 8), ("cached", C.c_int32)]


class gb_blocks(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("n_atoms_total", C.c_int64), ("val_nnz", C.c_int64),
                ("val_capacity", C.c_int64), ("atom_ptr", C.c_void_p), ("atoms", C.c_void_p),
                ("val_ptr", C.c_void_p), ("val", C.c_void_p)]


# every entry point declared in include/gbqr.h: (name, restype, argtypes)
SIGNATURES = [
    ("gb_create", C.c_int, [C.POINTER(C.c_void_p), C.c_void_p]),
    ("gb_destroy", C.c_int, [C.c_void_p]),
    ("gb_set_workspace", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("gb_required_workspace", C.c_size_t, [C.c_void_p]),
    ("gb_launch_count", C.c_int64, [C.c_void_p]),
    ("gb_status_string", C.c_char_p, [C.c_int]),
    ("gb_version", C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("gb_graph_build_workspace_size", C.c_size_t, [C.c_int32, C.c_int64, C.c_int64, C.c_int]),
    ("gb_graph_build", C.c_int, [C.c_void_p, C.POINTER(gb_csr), C.POINTER(gb_csc), C.c_double, C.c_int,
                                 C.POINTER(gb_graph)]),
    ("gb_partition_workspace_size", C.c_size_t, [C.c_int32, C.c_int64, C.c_int32]),
    ("gb_partition", C.c_int, [C.c_void_p, C.POINTER(gb_graph), C.c_void_p, C.c_int32, C.c_int32,
                               C.POINTER(gb_part)]),
    ("gb_partition_capped_workspace_size", C.c_size_t, [C.c_int32, C.c_int64, C.c_int32, C.c_int32]),
    ("gb_partition_capped", C.c_int, [C.c_void_p, C.POINTER(gb_graph), C.c_void_p, C.c_int32, C.c_void_p,
                                      C.c_int32, C.c_int32, C.POINTER(gb_part)]),
    ("gb_partition_noalloc_scratch_bytes", C.c_size_t, []),
    ("gb_partition_noalloc", C.c_int, [C.c_void_p, C.POINTER(gb_graph), C.c_void_p, C.c_int32, C.c_int32,
                                       C.POINTER(gb_part)]),
    ("gb_density_workspace_size", C.c_int, [C.POINTER(gb_part), C.c_int32, C.POINTER(gb_opts),
                                            C.POINTER(C.c_size_t)]),
    ("gb_density_and_response", C.c_int, [C.c_void_p, C.POINTER(gb_csr), C.POINTER(gb_csr), C.c_int32,
                                          C.c_double, C.c_double, C.POINTER(gb_part), C.POINTER(gb_opts),
                                          C.POINTER(C.c_double), C.POINTER(gb_csc), C.POINTER(gb_csc),
                                          C.POINTER(C.c_double), C.POINTER(gb_report)]),
    ("gb_mulliken_workspace_size", C.c_size_t, []),
    ("gb_mulliken_charges", C.c_int, [C.c_void_p, C.POINTER(gb_csc), C.POINTER(gb_csc), C.c_int32, C.c_int32,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("gb_preconditioner_workspace_size", C.c_size_t, [C.POINTER(gb_part)]),
    ("gb_preconditioner", C.c_int, [C.c_void_p, C.POINTER(gb_csr), C.POINTER(gb_part), C.c_double, C.c_double,
                                    C.POINTER(gb_csr), C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_double),
                                    C.POINTER(gb_blocks)]),
    ("gb_krylov_workspace_size", C.c_size_t, [C.POINTER(gb_csr), C.POINTER(gb_part), C.c_int32,
                                              C.POINTER(gb_opts)]),
    ("gb_krylov_update", C.c_int, [C.c_void_p, C.POINTER(gb_csr), C.POINTER(gb_part), C.c_double, C.c_double,
                                   C.POINTER(gb_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.POINTER(gb_blocks), C.c_double, C.c_int32, C.c_double,
                                   C.POINTER(gb_opts), C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    ("gb_last_device_error", C.c_int, [C.POINTER(C.c_char_p)]),
    ("gb_plan_autotune", C.c_int, [C.c_void_p, C.POINTER(gb_csr), C.POINTER(gb_csr), C.c_int32, C.c_double,
                                   C.c_double, C.POINTER(gb_part), C.POINTER(gb_opts), C.c_double,
                                   C.POINTER(gb_csc), C.POINTER(gb_csc), C.POINTER(gb_plan)]),
]

_lib = None


def load() -> C.CDLL:
    """Load libgbqr.so (built by paper_2212_01997_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(func: str, status: int):
    if status != GB_OK:
        raise GbError(func, status)
