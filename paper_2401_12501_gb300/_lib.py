"""ctypes binding of libparametrix.so (argument marshalling only).

Every function here converts Python arguments to the C ABI declared in
include/parametrix.h and raises on a non-zero status.  All computation runs
in the CUDA library; if the library has not been built this module raises
at import time instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PM_LIBRARY selects another build of the library (e.g. libparametrix_checked.so)
LIB_PATH = os.environ.get("PM_LIBRARY") or os.path.join(_HERE, "libparametrix.so")

PM_OK = 0
PM_ERR_TIMEOUT = 7
PM_PREC_FP64, PM_PREC_FP32, PM_PREC_FP32_TC, PM_PREC_FF, PM_PREC_FMM = 0, 1, 2, 3, 4
PM_PART_SMOOTH_R, PM_PART_SMOOTH_K, PM_PART_NEAR_R, PM_PART_NEAR_K = 0, 1, 2, 3
PM_SOLVE_PROJECT_RHS = 1
PM_SOLVE_DEVICE_PTRS = 2
PM_SOLVE_INITIAL_GUESS = 4
PM_BVP_NEUMANN, PM_BVP_DIRICHLET = 0, 1

STATUS_NAMES = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_OOM", 3: "PM_ERR_CUDA",
                4: "PM_ERR_NOT_CONVERGED", 5: "PM_ERR_BREAKDOWN",
                6: "PM_ERR_RHS_NOT_MEAN_ZERO", 7: "PM_ERR_TIMEOUT", 8: "PM_ERR_INTERNAL",
                9: "PM_ERR_NO_COEFF"}

# every symbol include/parametrix.h declares
EXPORTS = ["pm_default_opts", "pm_ctx_create", "pm_ctx_destroy", "pm_surface_create",
           "pm_surface_destroy", "pm_surface_info", "pm_surface_set_coeff", "pm_apply_R",
           "pm_apply_K", "pm_apply_part", "pm_surface_get_near", "pm_solve",
           "pm_status_str", "pm_last_error", "pm_profile_enable", "pm_profile_read",
           "pm_surface_tune", "pm_selftest_fflog", "pm_smooth_remainder_f32_noalloc",
           "pm_surface_fmm_stats", "pm_server_create", "pm_server_destroy", "pm_server_submit",
           "pm_server_poll", "pm_server_wait", "pm_server_stats", "pm_server_submit_desc",
           "pm_server_wait_ex", "pm_server_stats_ex", "pm_server_configure", "pm_solve_multi", "pm_surface_set_knobs",
           "pm_surface_get_knobs", "pm_surface_autotune", "pm_ctx_info", "pm_surface_clone",
           "pm_selftest_fmm_classes", "pm_selftest_tc_gemm", "pm_selftest_green",
           "pm_selftest_green_f32", "pm_selftest_smooth_c_f32", "pm_smooth_c_f32",
           "pm_surface_set_coeff_c", "pm_apply_c", "pm_solve_c", "pm_surface_create_tri",
           "pm_selftest_tri_basis", "pm_surface_check", "pm_selftest_green_c",
           "pm_surface_store_ff", "pm_surface_stored_ff", "pm_bvp_create", "pm_bvp_destroy",
           "pm_bvp_apply", "pm_bvp_solve"]
(PM_PHASE_PREP, PM_PHASE_DIRECT_R, PM_PHASE_DIRECT_K, PM_PHASE_NEAR, PM_PHASE_SOLVE_VEC,
 PM_PHASE_DIRECT64, PM_PHASE_FMM_M2L, PM_PHASE_FMM_P2P, PM_PHASE_DIRECT64_K,
 PM_PHASE_COUNT) = range(10)


class PmOpts(C.Structure):
    _fields_ = [("near_factor", C.c_double), ("theta_tol", C.c_double),
                ("theta_max_width", C.c_double), ("near_eta", C.c_double),
                ("near_max_depth", C.c_int), ("near_max_leaves", C.c_int),
                ("gmres_restart", C.c_int), ("max_refine", C.c_int),
                ("inner_tol", C.c_double), ("mean_tol", C.c_double),
                ("residual_prec", C.c_int), ("fmm_depth", C.c_int), ("batch_rhs", C.c_int),
                ("direct_tpt", C.c_int),
                ("direct_blocks_per_sm", C.c_int), ("direct_symmetric", C.c_int),
                ("residual_update", C.c_int), ("fmm_tensor_m2l", C.c_int)]


class PmSolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int),
                ("residual", C.c_double), ("removed_mean", C.c_double),
                ("seconds", C.c_double), ("residual_updates", C.c_int)]


class PmKnobs(C.Structure):
    _fields_ = [("direct_tpt", C.c_int), ("direct_blocks_per_sm", C.c_int),
                ("batch_rhs_per_block", C.c_int), ("batch_blocks_per_sm", C.c_int),
                ("fmm_depth", C.c_int), ("fmm_streams", C.c_int)]


class PmTuneResult(C.Structure):
    _fields_ = [("best", PmKnobs), ("best_ms", C.c_double), ("default_ms", C.c_double),
                ("candidates", C.c_int)]


class PmRequestTimes(C.Structure):
    _fields_ = [("latency_s", C.c_double), ("build_s", C.c_double), ("solve_s", C.c_double),
                ("queue_s", C.c_double)]


class PmOperatorDesc(C.Structure):
    _fields_ = [("geometry_id", C.c_ulonglong), ("coeff_id", C.c_ulonglong),
                ("npatch", C.c_int), ("p", C.c_int),
                ("nodes", C.c_void_p), ("normals", C.c_void_p), ("tangents", C.c_void_p),
                ("curvature", C.c_void_p), ("weights", C.c_void_p), ("a", C.c_void_p),
                ("grad_a", C.c_void_p), ("opts", C.POINTER(PmOpts))]


class PmError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.pm_default_opts.argtypes = [C.POINTER(PmOpts)]
    lib.pm_default_opts.restype = None
    lib.pm_ctx_create.argtypes = [C.c_int, C.POINTER(P)]
    lib.pm_ctx_destroy.argtypes = [P]
    lib.pm_ctx_destroy.restype = None
    lib.pm_surface_create.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P,
                                      C.POINTER(PmOpts), C.POINTER(P)]
    lib.pm_surface_destroy.argtypes = [P]
    lib.pm_surface_clone.argtypes = [P, C.POINTER(P)]
    lib.pm_selftest_fmm_classes.argtypes = [P, P, P]
    lib.pm_selftest_tc_gemm.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.POINTER(C.c_double)]
    lib.pm_selftest_green.argtypes = [P, C.c_int, C.c_double, P]
    lib.pm_selftest_green_f32.argtypes = [P, C.c_int, C.c_float, P]
    lib.pm_selftest_smooth_c_f32.argtypes = [C.c_int, P, P, P, P, P, P, P, P]
    lib.pm_smooth_c_f32.argtypes = [C.c_int, P, P, P, P, P, P, P, P, P]
    lib.pm_surface_destroy.restype = None
    lib.pm_surface_tune.argtypes = [P, C.c_int, C.c_int]
    lib.pm_surface_set_knobs.argtypes = [P, C.POINTER(PmKnobs)]
    lib.pm_surface_get_knobs.argtypes = [P, C.POINTER(PmKnobs)]
    lib.pm_surface_autotune.argtypes = [P, C.c_int, C.c_int, C.c_int, C.POINTER(PmTuneResult)]
    lib.pm_ctx_info.argtypes = [P, C.c_char_p, C.c_int, C.POINTER(C.c_int)]
    lib.pm_surface_fmm_stats.argtypes = [P, P]
    lib.pm_server_create.argtypes = [P, C.c_size_t, C.c_int, C.c_int, C.POINTER(P)]
    lib.pm_server_destroy.argtypes = [P]
    lib.pm_server_destroy.restype = None
    lib.pm_server_submit.argtypes = [P, P, P, C.c_double, C.c_int, C.POINTER(C.c_ulonglong)]
    lib.pm_server_poll.argtypes = [P, C.c_ulonglong, C.POINTER(C.c_int)]
    lib.pm_server_wait.argtypes = [P, C.c_ulonglong, P, C.POINTER(PmSolveInfo),
                                   C.POINTER(C.c_double), C.c_int]
    lib.pm_server_stats.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                    C.POINTER(C.c_longlong), C.POINTER(C.c_size_t)]
    lib.pm_server_submit_desc.argtypes = [P, C.POINTER(PmOperatorDesc), P, C.c_double, C.c_int,
                                          C.POINTER(C.c_ulonglong)]
    lib.pm_server_wait_ex.argtypes = [P, C.c_ulonglong, P, C.POINTER(PmSolveInfo),
                                      C.POINTER(PmRequestTimes), C.c_int]
    lib.pm_server_configure.argtypes = [P, C.c_int, C.c_int]
    lib.pm_server_stats_ex.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_size_t),
                                       C.POINTER(C.c_size_t), C.POINTER(C.c_int)]
    lib.pm_selftest_fflog.argtypes = [P, P, P, C.c_int, P]
    lib.pm_smooth_remainder_f32_noalloc.argtypes = [C.c_int, P, P, P, P, P, P, P, P]
    lib.pm_surface_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.pm_surface_set_coeff.argtypes = [P, P, P]
    lib.pm_surface_set_coeff_c.argtypes = [P, P, P, P]
    lib.pm_surface_create_tri.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P, P, P, C.POINTER(P)]
    lib.pm_selftest_tri_basis.argtypes = [C.c_int, P, C.c_int, P, P, P, P, P]
    lib.pm_surface_check.argtypes = [P]
    lib.pm_surface_store_ff.argtypes = [P, C.c_int]
    lib.pm_surface_stored_ff.argtypes = [P]
    lib.pm_surface_stored_ff.restype = C.c_int
    lib.pm_bvp_create.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                  C.POINTER(P)]
    lib.pm_bvp_destroy.argtypes = [P]
    lib.pm_bvp_destroy.restype = None
    lib.pm_bvp_apply.argtypes = [P, P, P, P, P]
    lib.pm_bvp_solve.argtypes = [P, P, P, C.c_double, C.c_int, P, P, P, C.POINTER(PmSolveInfo)]
    lib.pm_selftest_green_c.argtypes = [P, C.c_int, C.c_double, C.c_double, P]
    lib.pm_apply_c.argtypes = [P, C.c_int, P, P, C.c_int, P]
    lib.pm_solve_c.argtypes = [P, P, P, C.c_double, C.c_int, P, C.POINTER(PmSolveInfo)]
    for name in ("pm_apply_R", "pm_apply_K"):
        getattr(lib, name).argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, P]
    lib.pm_apply_part.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int, C.c_int, P]
    lib.pm_surface_get_near.argtypes = [P, P, P, P, P]
    lib.pm_solve.argtypes = [P, P, P, C.c_int, C.c_double, C.c_int, C.c_int, C.c_uint,
                             P, C.POINTER(PmSolveInfo), P]
    lib.pm_solve_multi.argtypes = [C.POINTER(P), C.c_int, C.POINTER(C.c_int), C.POINTER(P),
                                   C.POINTER(P), C.c_double, C.c_int, C.c_int, C.c_uint,
                                   C.POINTER(PmSolveInfo), P]
    lib.pm_profile_enable.argtypes = [P, C.c_int]
    lib.pm_profile_read.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int]
    lib.pm_status_str.argtypes = [C.c_int]
    lib.pm_status_str.restype = C.c_char_p
    lib.pm_last_error.argtypes = []
    lib.pm_last_error.restype = C.c_char_p
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def check(status: int, where: str):
    if status != PM_OK:
        msg = lib().pm_last_error().decode(errors="replace")
        raise PmError(status, where, msg)


def ptr(a) -> C.c_void_p:
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return C.c_void_p(None)
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer type {type(a)}")


def default_opts() -> PmOpts:
    o = PmOpts()
    lib().pm_default_opts(C.byref(o))
    return o
