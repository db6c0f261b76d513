"""ctypes declarations of the C-ABI in include/mcx.h.

Loading never falls back to anything: if the compiled library is missing the
import fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmcx.so")

# Every symbol declared in include/mcx.h; the library must export all of them.
EXPORTS = (
    "mcx_plan_create",
    "mcx_plan_get_info",
    "mcx_estimate",
    "mcx_expm_multiply",
    "mcx_estimate_rqmc",
    "mcx_estimate_level_difference",
    "mcx_combine_levels",
    "mcx_gather_rate",
    "mcx_estimate_noalloc",
    "mcx_estimate_forward",
    "mcx_trace_forward",
    "mcx_total_communicability",
    "mcx_trace_paths",
    "mcx_power_iteration",
    "mcx_plan_export",
    "mcx_sync",
    "mcx_plan_destroy",
    "mcx_status_string",
    "mcx_version",
    "mcx_batch_create",
    "mcx_batch_run",
    "mcx_batch_result",
    "mcx_batch_set_v",
    "mcx_batch_get_info",
    "mcx_batch_sync",
    "mcx_batch_destroy",
    "mcx_cv_prepare",
    "mcx_cv_targets",
    "mcx_mlp_create",
    "mcx_mlp_set",
    "mcx_mlp_get",
    "mcx_mlp_predict",
    "mcx_mlp_sync",
    "mcx_mlp_gradient",
    "mcx_mlp_fit",
    "mcx_mlp_destroy",
    "mcx_cv_coefficients",
    "mcx_estimate_cv",
    "mcx_cvbatch_create",
    "mcx_cvbatch_set_paths",
    "mcx_cvbatch_run",
    "mcx_cvbatch_result",
    "mcx_cvbatch_coefficients",
    "mcx_cvbatch_get_info",
    "mcx_cvbatch_sync",
    "mcx_cvbatch_destroy",
    "mcx_debug_fail_alloc",
    "mcx_debug_pool_usage",
    "mcx_debug_mlp_wait_polls",
)

MCX_OK = 0
STATUS_NAMES = {
    0: "MCX_OK", -1: "MCX_E_INVALID", -2: "MCX_E_NEG_OFFDIAG", -3: "MCX_E_NONFINITE", -4: "MCX_E_NEG_V",
    -5: "MCX_E_CUDA", -6: "MCX_E_OOM", -7: "MCX_E_TIMEOUT", -8: "MCX_E_UNSUPPORTED", -9: "MCX_E_OVERFLOW",
}
FUNCTIONALS = {"exact": 0, "strang": 1, "lie": 2}
PRECISIONS = {"fp32": 0, "fp64": 1}
PLAN_HOST_INPUT = 0x1


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nnz_off", C.c_int64), ("weighted_rows", C.c_int64),
                ("max_deg", C.c_int32), ("reserved", C.c_int32), ("device_bytes", C.c_int64)]


class Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("v", C.c_void_p), ("n_times", C.c_int32), ("times", C.c_void_p),
                ("paths", C.c_uint64)]


class BatchInfo(C.Structure):
    _fields_ = [("problems", C.c_int32), ("pairs", C.c_int32), ("states", C.c_int64), ("total_paths", C.c_uint64),
                ("work_items", C.c_uint32), ("chunk", C.c_uint32), ("blocks_per_sm", C.c_int32),
                ("grid", C.c_int32), ("count_deposits", C.c_int32), ("lane_refill", C.c_int32),
                ("tuned_ms", C.c_double)]


class CvProblem(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("n_rhs", C.c_int32), ("v", C.c_void_p), ("t", C.c_void_p),
                ("paths", C.c_uint64)]


class CvBatchInfo(C.Structure):
    _fields_ = [("problems", C.c_int32), ("pairs", C.c_int32), ("states", C.c_int64), ("total_paths", C.c_uint64),
                ("work_items", C.c_uint32), ("chunk", C.c_uint32), ("blocks_per_sm", C.c_int32),
                ("grid", C.c_int32), ("staged", C.c_int32), ("control", C.c_int32), ("tuned_ms", C.c_double)]


CV_CONTROLS = {"none": 0, "taylor": 1, "learned": 2}


class Stats(C.Structure):
    _fields_ = [("paths", C.c_uint64), ("jumps", C.c_uint64), ("status_bits", C.c_uint32),
                ("reserved", C.c_uint32)]


class MCXError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({status_string(code)})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libmcx.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"mcx CUDA library not built: {path} is missing "
                          "(run `python -m paper_1904_12759_gb300.build` or __graft_entry__.build())")
    L = C.CDLL(path)
    vp, i64, u64, i32, u32, dbl, st = C.c_void_p, C.c_int64, C.c_uint64, C.c_int32, C.c_uint32, C.c_double, C.c_int
    L.mcx_plan_create.argtypes = [i64, i64, vp, vp, vp, u32, vp, C.POINTER(vp)]
    L.mcx_plan_create.restype = st
    L.mcx_plan_get_info.argtypes = [vp, C.POINTER(PlanInfo)]
    L.mcx_plan_get_info.restype = st
    L.mcx_estimate.argtypes = [vp, vp, dbl, C.c_int, i32, u64, vp, i64, u64, u64, C.c_int, vp, vp, vp]
    L.mcx_estimate.restype = st
    L.mcx_expm_multiply.argtypes = [i64, i64, vp, vp, vp, vp, dbl, dbl, C.c_int, i32, u64, vp, i64, u64, u64,
                                    C.c_int, u32, vp, vp, C.POINTER(dbl), vp]
    L.mcx_expm_multiply.restype = st
    L.mcx_estimate_rqmc.argtypes = [vp, vp, dbl, C.c_int, i32, u32, u32, u32, vp, i64, u64, C.c_int, vp, vp, vp]
    L.mcx_estimate_rqmc.restype = st
    L.mcx_estimate_level_difference.argtypes = [vp, vp, dbl, C.c_int, i32, u64, vp, i64, u64, u64, C.c_int, vp,
                                                vp, vp]
    L.mcx_estimate_level_difference.restype = st
    L.mcx_combine_levels.argtypes = [i32, i64, vp, vp, vp, vp, vp]
    L.mcx_combine_levels.restype = st
    L.mcx_gather_rate.argtypes = [u64, C.c_int, u64, C.POINTER(dbl), vp]
    L.mcx_gather_rate.restype = st
    L.mcx_estimate_noalloc.argtypes = [vp, vp, dbl, C.c_int, i32, u64, vp, i64, u64, u64, C.c_int, vp, vp, vp]
    L.mcx_estimate_noalloc.restype = st
    L.mcx_estimate_forward.argtypes = [vp, vp, dbl, C.c_int, i32, u64, u64, u64, C.c_int, vp, vp, vp]
    L.mcx_estimate_forward.restype = st
    L.mcx_trace_forward.argtypes = [vp, vp, dbl, C.c_int, i32, u64, u64, u32, C.c_int, vp, vp, vp, vp, vp, vp]
    L.mcx_trace_forward.restype = st
    L.mcx_total_communicability.argtypes = [vp, dbl, C.c_int, i32, u64, u64, u64, C.c_int, vp, vp, vp]
    L.mcx_total_communicability.restype = st
    L.mcx_trace_paths.argtypes = [vp, dbl, C.c_int, i32, i32, u64, u64, u32, C.c_int, vp, vp, vp, vp, vp]
    L.mcx_trace_paths.restype = st
    L.mcx_power_iteration.argtypes = [i64, vp, vp, vp, i32, dbl, vp, C.POINTER(dbl), C.POINTER(i32), vp]
    L.mcx_power_iteration.restype = st
    L.mcx_plan_export.argtypes = [vp] + [vp] * 10 + [vp]
    L.mcx_plan_export.restype = st
    L.mcx_sync.argtypes = [vp, vp, C.POINTER(Stats)]
    L.mcx_sync.restype = st
    L.mcx_plan_destroy.argtypes = [vp]
    L.mcx_plan_destroy.restype = None
    L.mcx_batch_create.argtypes = [i32, C.POINTER(Problem), C.c_char_p, vp, C.POINTER(vp)]
    L.mcx_batch_create.restype = st
    L.mcx_batch_run.argtypes = [vp, u64, vp]
    L.mcx_batch_run.restype = st
    L.mcx_batch_result.argtypes = [vp, i32, i32, vp, vp, vp]
    L.mcx_batch_result.restype = st
    L.mcx_batch_set_v.argtypes = [vp, i32, vp, vp]
    L.mcx_batch_set_v.restype = st
    L.mcx_batch_get_info.argtypes = [vp, C.POINTER(BatchInfo)]
    L.mcx_batch_get_info.restype = st
    L.mcx_batch_sync.argtypes = [vp, vp, C.POINTER(Stats)]
    L.mcx_batch_sync.restype = st
    L.mcx_batch_destroy.argtypes = [vp]
    L.mcx_batch_destroy.restype = None
    L.mcx_cv_prepare.argtypes = [i64, vp, vp, vp, vp, dbl, vp, vp, vp, vp]
    L.mcx_cv_prepare.restype = st
    L.mcx_cv_targets.argtypes = [i64, vp, vp, dbl, vp, vp]
    L.mcx_cv_targets.restype = st
    L.mcx_mlp_create.argtypes = [u64, C.POINTER(vp)]
    L.mcx_mlp_create.restype = st
    L.mcx_mlp_set.argtypes = [vp, vp, vp, vp]
    L.mcx_mlp_set.restype = st
    L.mcx_mlp_get.argtypes = [vp, vp, vp, vp]
    L.mcx_mlp_get.restype = st
    L.mcx_mlp_predict.argtypes = [vp, i64, vp, vp, vp]
    L.mcx_mlp_predict.restype = st
    L.mcx_mlp_sync.argtypes = [vp, vp]
    L.mcx_mlp_sync.restype = st
    L.mcx_mlp_gradient.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.mcx_mlp_gradient.restype = st
    L.mcx_mlp_fit.argtypes = [vp, i64, vp, vp, i32, i32, C.c_float, u64, vp, vp]
    L.mcx_mlp_fit.restype = st
    L.mcx_mlp_destroy.argtypes = [vp]
    L.mcx_mlp_destroy.restype = None
    L.mcx_cv_coefficients.argtypes = [i64, vp, vp, vp, vp, vp, dbl, vp, vp, vp]
    L.mcx_cv_coefficients.restype = st
    L.mcx_estimate_cv.argtypes = [vp, vp, dbl, u64, vp, i64, u64, u64, C.c_int, vp, vp, vp]
    L.mcx_estimate_cv.restype = st
    L.mcx_cvbatch_create.argtypes = [i32, C.POINTER(CvProblem), C.c_int, vp, C.c_int, C.c_char_p, vp,
                                     C.POINTER(vp)]
    L.mcx_cvbatch_create.restype = st
    L.mcx_cvbatch_set_paths.argtypes = [vp, vp, vp]
    L.mcx_cvbatch_set_paths.restype = st
    L.mcx_cvbatch_run.argtypes = [vp, u64, vp]
    L.mcx_cvbatch_run.restype = st
    L.mcx_cvbatch_result.argtypes = [vp, i32, i32, vp, vp, vp]
    L.mcx_cvbatch_result.restype = st
    L.mcx_cvbatch_coefficients.argtypes = [vp, i32, i32, vp, vp]
    L.mcx_cvbatch_coefficients.restype = st
    L.mcx_cvbatch_get_info.argtypes = [vp, C.POINTER(CvBatchInfo)]
    L.mcx_cvbatch_get_info.restype = st
    L.mcx_cvbatch_sync.argtypes = [vp, vp, C.POINTER(Stats)]
    L.mcx_cvbatch_sync.restype = st
    L.mcx_cvbatch_destroy.argtypes = [vp]
    L.mcx_cvbatch_destroy.restype = None
    L.mcx_debug_fail_alloc.argtypes = [i64]
    L.mcx_debug_fail_alloc.restype = i64
    L.mcx_debug_pool_usage.argtypes = [C.POINTER(u64), C.POINTER(u64)]
    L.mcx_debug_pool_usage.restype = st
    L.mcx_debug_mlp_wait_polls.argtypes = [vp, u32]
    L.mcx_debug_mlp_wait_polls.restype = st
    L.mcx_status_string.argtypes = [C.c_int]
    L.mcx_status_string.restype = C.c_char_p
    L.mcx_version.restype = C.c_int
    _lib = L
    return L


def status_string(code: int) -> str:
    try:
        return load().mcx_status_string(int(code)).decode()
    except ImportError:
        return STATUS_NAMES.get(code, str(code))


def check(code: int, where: str) -> None:
    if code != MCX_OK:
        raise MCXError(code, where)
