"""ctypes declarations of the C ABI in ``include/grape_hg.h`` (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

from .build import LIB, build_library

GRAPE_CSR, GRAPE_DENSE = 0, 1
GRAPE_FP64, GRAPE_FP32_BULK, GRAPE_TC_FP16, GRAPE_TC_BF16 = 0, 1, 2, 3
GRAPE_PROP_TAYLOR, GRAPE_PROP_EIG = 0, 1

STATUS = {
    0: "GRAPE_OK", 1: "GRAPE_EINVAL", 2: "GRAPE_ENOMEM", 3: "GRAPE_ECUDA", 4: "GRAPE_ETOL",
    5: "GRAPE_ETIMEOUT", 6: "GRAPE_ENOTHERMITIAN", 7: "GRAPE_ESTATE", 8: "GRAPE_ENONFINITE",
}

# Every symbol include/grape_hg.h declares.
EXPORTED = [
    "grape_problem_create", "grape_problem_destroy", "grape_cost_and_grad", "grape_cost", "grape_grad",
    "grape_sync_status", "grape_problem_info", "grape_step_schedule", "grape_select_ms", "grape_error_bound",
    "grape_status_string", "grape_last_error", "grape_abi_version", "grape_taylor_step_noalloc",
    "grape_batch_create", "grape_batch_destroy", "grape_batch_cost_and_grad", "grape_batch_info", "grape_optimize",
    "grape_set_kernel_tracing", "grape_kernel_times", "grape_fp64_fma_rate",
]

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class GrapeOp(C.Structure):
    _fields_ = [("fmt", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.POINTER(C.c_int64)),
                ("colind", C.POINTER(C.c_int32)), ("values", C.POINTER(C.c_double))]


class GrapeDesc(C.Structure):
    _fields_ = [("dim", C.c_int64), ("n_controls", C.c_int32), ("n_steps", C.c_int32), ("n_states", C.c_int32),
                ("dt", C.c_double), ("H0", GrapeOp), ("Hk", C.POINTER(GrapeOp)),
                ("psi0", C.POINTER(C.c_double)), ("target", C.POINTER(C.c_double)),
                ("omega_diag", C.POINTER(C.c_double)),
                ("w_fid", C.c_double), ("w_forbid", C.c_double), ("w_amp", C.c_double),
                ("tau", C.c_double), ("m_max", C.c_int32), ("ckpt_every", C.c_int32), ("precision", C.c_int32),
                ("cluster", C.c_int32), ("device", C.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p), ("backward_mode", C.c_int32),
                ("bulk_norm_cap", C.c_double), ("w_tint", C.c_double), ("propagator", C.c_int32),
                ("grad_cluster", C.c_int32), ("block_steps", C.c_int32)]


class GrapeInfo(C.Structure):
    _fields_ = [("device_bytes", C.c_int64), ("union_nnz", C.c_int64), ("ctrl_entries", C.c_int64),
                ("sigma", C.c_int32), ("m_cap", C.c_int32), ("s_cap", C.c_int32), ("cluster", C.c_int32),
                ("ckpt_every", C.c_int32), ("smem_bytes", C.c_int32), ("total_terms", C.c_int64),
                ("max_norm", C.c_double), ("backward_mode", C.c_int32), ("cluster_forward", C.c_int32),
                ("propagator", C.c_int32), ("grad_cluster", C.c_int32), ("block_steps", C.c_int32),
                ("fused_fallback", C.c_int32)]


class GrapeBatchInfo(C.Structure):
    _fields_ = [("members", C.c_int32), ("queued", C.c_int32), ("queue_items", C.c_int32), ("queue_ctas", C.c_int32),
                ("lanes", C.c_int32), ("lane_members", C.c_int32)]


class GrapeKernelTimes(C.Structure):
    _fields_ = [("launches", C.c_int32 * 5), ("ms", C.c_double * 5)]


_LIB = None


def lib(path: str | None = None):
    """Load libgrape_hg.so (building it first if it is missing or stale); raises if that is impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = build_library()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    P = C.c_void_p
    L.grape_problem_create.argtypes = [C.POINTER(GrapeDesc), C.POINTER(P)]
    L.grape_problem_create.restype = C.c_int
    L.grape_problem_destroy.argtypes = [P]
    L.grape_problem_destroy.restype = None
    L.grape_cost_and_grad.argtypes = [P, P, P, P, C.c_int32, P]
    L.grape_cost_and_grad.restype = C.c_int
    L.grape_cost.argtypes = [P, P, P, C.c_int32, P]
    L.grape_cost.restype = C.c_int
    L.grape_grad.argtypes = [P, P, C.c_int32, P]
    L.grape_grad.restype = C.c_int
    L.grape_sync_status.argtypes = [P, P]
    L.grape_sync_status.restype = C.c_int
    L.grape_problem_info.argtypes = [P, C.POINTER(GrapeInfo)]
    L.grape_problem_info.restype = C.c_int
    L.grape_step_schedule.argtypes = [P, P, P, P]
    L.grape_step_schedule.restype = C.c_int
    L.grape_select_ms.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.grape_select_ms.restype = C.c_int
    L.grape_error_bound.argtypes = [C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.grape_error_bound.restype = C.c_double
    L.grape_taylor_step_noalloc.argtypes = [C.c_int64, C.c_int64, C.c_int32, P, P, P, C.c_double, C.c_int32, C.c_int32, P, P, P]
    L.grape_taylor_step_noalloc.restype = C.c_int
    L.grape_batch_create.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32, C.POINTER(P), C.POINTER(P)]
    L.grape_batch_create.restype = C.c_int
    L.grape_batch_info.argtypes = [P, C.POINTER(GrapeBatchInfo)]
    L.grape_batch_info.restype = C.c_int
    L.grape_batch_destroy.argtypes = [P]
    L.grape_batch_destroy.restype = None
    L.grape_batch_cost_and_grad.argtypes = [P, C.POINTER(P), P, C.POINTER(P), C.c_int32, P]
    L.grape_batch_cost_and_grad.restype = C.c_int
    L.grape_optimize.argtypes = [P, P, C.c_int32, C.c_double, P, C.c_int32, P]
    L.grape_optimize.restype = C.c_int
    L.grape_set_kernel_tracing.argtypes = [P, C.c_int32]
    L.grape_set_kernel_tracing.restype = C.c_int
    L.grape_kernel_times.argtypes = [P, C.POINTER(GrapeKernelTimes)]
    L.grape_kernel_times.restype = C.c_int
    L.grape_fp64_fma_rate.argtypes = [C.c_int32, C.POINTER(C.c_double)]
    L.grape_fp64_fma_rate.restype = C.c_int
    L.grape_status_string.argtypes = [C.c_int]
    L.grape_status_string.restype = C.c_char_p
    L.grape_last_error.argtypes = []
    L.grape_last_error.restype = C.c_char_p
    L.grape_abi_version.argtypes = []
    L.grape_abi_version.restype = C.c_int32
    _LIB = L
    return L


class GrapeError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().grape_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


def check(status: int, where: str):
    if status != 0:
        raise GrapeError(status, where)
