"""ctypes view of ``libcegpu.so`` (the C ABI declared in include/ce.h).

Only argument marshalling lives here.  Loading fails loudly when the library
is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcegpu.so")

CE_OK = 0
CE_ERR_INVALID_ARG = 1
CE_ERR_NOT_SPD = 2
CE_ERR_NO_CONVERGENCE = 3
CE_ERR_OOM = 4
CE_ERR_CUDA = 5
CE_ERR_LIMIT = 6
CE_TOL_REL = 0
CE_TOL_ABS = 1
CE_TOL_FIXED = 2
CE_PREC_FP64 = 0
CE_PREC_FP32 = 1
CE_RANK_SVD = 0
CE_RANK_LEARNED = 1


class ce_opts(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("tol_mode", C.c_int),
        ("levels", C.c_int),
        ("J", C.c_int),
        ("precision", C.c_int),
        ("coloring", C.c_int),
        ("stream", C.c_void_p),
        ("rank_mode", C.c_int),
        ("rank_model", C.c_void_p),
        ("oversample", C.c_int),
        ("seed", C.c_uint64),
        ("row_shape", C.c_int),
        ("rank", C.c_int),
        ("nmax", C.c_int),
        ("record_features", C.c_int),
        ("gemm_engine", C.c_int),
    ]


class ce_info(C.Structure):
    _fields_ = [
        ("levels_done", C.c_int),
        ("err_level", C.c_int),
        ("err_block", C.c_int),
        ("err_reason", C.c_int),
        ("err_pivot", C.c_int),
        ("err_value", C.c_double),
        ("coarse_n", C.c_int),
        ("factor_bytes", C.c_int64),
        ("blocks", C.c_int * 16),
        ("colours", C.c_int * 16),
        ("max_block", C.c_int * 16),
        ("level_ms", C.c_double * 16),
        ("level_flops", C.c_double * 16),
        ("level_bytes", C.c_double * 16),
        ("coarse_ms", C.c_double),
        ("learned_rows", C.c_int * 16),
        ("fallback_rows", C.c_int * 16),
        ("host_ms", C.c_double * 16),
        ("total_ms", C.c_double),
        ("row_shape", C.c_int * 16),
        ("row_learned", C.c_int * 16),
        ("spec_miss", C.c_int * 16),
        ("big_rows", C.c_int * 16),
        ("big_ms", C.c_double * 8),
        ("jacobi_capped", C.c_int * 16),
        ("row_phase_ms", (C.c_double * 12) * 16),
        ("jacobi_sweeps", (C.c_double * 2) * 16),
    ]


class ce_pcg_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres", C.c_double), ("converged", C.c_int)]


P = C.c_void_p
PP = C.POINTER(C.c_void_p)
I64P = C.POINTER(C.c_int64)
I32P = C.POINTER(C.c_int32)
DP = C.POINTER(C.c_double)
FP = C.c_void_p

# name -> (restype, argtypes); every extern "C" function of include/ce.h
SIGNATURES = {
    "ce_opts_default": (None, [C.POINTER(ce_opts)]),
    "csb_build": (C.c_int, [C.c_int64, I64P, I32P, DP, I32P, C.c_int32, PP]),
    "csb_build_batched": (C.c_int, [C.c_int, I64P, I64P, I32P, DP, I32P, I32P, PP]),
    "csb_update_values": (C.c_int, [P, DP, P]),
    "ce_plan_colours": (C.c_int, [C.c_int64, I64P, I32P, I32P, C.c_int32, C.c_int, I32P, C.POINTER(C.c_int)]),
    "ce_plan_level1_deps": (C.c_int, [C.c_int64, I64P, I32P, I32P, C.c_int32, I64P, I32P, C.c_int64,
                                      I64P]),
    "ce_plan_next_level": (C.c_int, [C.c_int64, I64P, I32P, I32P, C.c_int32, I32P, C.c_int, C.c_int, I32P,
                                     I32P, C.POINTER(C.c_int), I64P]),
    "ce_plan_level1_work": (C.c_int, [C.c_int64, I64P, I32P, I32P, C.c_int32, I32P, C.c_int, DP, DP]),
    "ce_plan_groups": (C.c_int, [C.c_int, I32P, C.c_int, C.c_int, I32P, C.POINTER(C.c_int)]),
    "ce_factorize_batched": (C.c_int, [P, C.POINTER(ce_opts), PP, C.POINTER(ce_info)]),
    "ce_factorize": (C.c_int, [P, C.POINTER(ce_opts), PP, C.POINTER(ce_info)]),
    "ce_factorize_simple": (C.c_int, [C.c_int64, I64P, I32P, DP, I32P, C.c_int32,
                                      C.c_double, C.c_int, PP]),
    "ce_apply": (C.c_int, [P, P, P, P]),
    "ce_autotune": (C.c_int, [P, C.POINTER(ce_opts), DP]),
    "pcg_solve": (C.c_int, [P, P, P, P, C.c_double, C.c_int, C.POINTER(ce_pcg_info), P]),
    "pcg_solve_batched": (C.c_int, [P, P, P, P, C.c_double, C.c_int, I32P, DP, I32P,
                                    C.POINTER(ce_pcg_info), P]),
    "pcg_solve_noalloc": (C.c_int, [P, P, P, P, C.c_double, C.c_int, C.POINTER(ce_pcg_info), P]),
    "ce_debug_svd": (C.c_int, [C.c_int, C.c_int, C.c_int, P, P, C.c_double, P, P, C.POINTER(C.c_int), P]),
    "minres_solve": (C.c_int, [P, P, P, P, C.c_double, C.c_int, C.POINTER(ce_pcg_info), P]),
    "ce_csb_destroy": (None, [P]),
    "ce_factor_destroy": (None, [P]),
    "ce_strerror": (C.c_char_p, [C.c_int]),
    "ce_last_error": (C.c_char_p, []),
    "ce_launch_count": (C.c_int64, []),
    "ce_measure_peak": (C.c_int, [C.c_int, DP, P]),
    "ce_mlp_nparams": (C.c_int, []),
    "ce_mlp_nfeatures": (C.c_int, []),
    "ce_mlp_init": (C.c_int, [FP, C.c_uint64, P]),
    "ce_mlp_grad": (C.c_int, [P, P, C.c_int, P, P, P]),
    "ce_mlp_train": (C.c_int, [P, P, C.c_int, P, C.c_int, C.c_float, DP, P]),
    "ce_mlp_pack": (C.c_int, [P, P, P]),
    "ce_mlp_predict": (C.c_int, [P, C.c_int, P, P, P]),
    "ce_factor_levels": (C.c_int, [P]),
    "ce_factor_level_size": (C.c_int, [P, C.c_int]),
    "ce_factor_get_level": (C.c_int, [P, C.c_int, I32P, I32P, I32P, DP]),
    "ce_factor_get_sigma": (C.c_int, [P, C.c_int, DP]),
    "ce_factor_get_features": (C.c_int, [P, C.c_int, FP, I32P]),
    "csb_blocks": (C.c_int, [P]),
    "csb_get_tuning": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_int), I32P, I32P]),
    "csb_set_tuning": (C.c_int, [P, C.c_int, C.c_int, C.c_int, I32P, I32P]),
    "ce_debug_wait_expiry": (C.c_int, [C.c_int, C.c_double, I32P, P]),
    "ce_debug_gemm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_int, C.c_int, P, C.c_int, C.c_int,
                                P, C.c_int, C.c_int, C.c_double, C.c_double, P]),
    "ce_plan_level1": (C.c_int, [C.c_int64, I64P, I32P, I32P, C.c_int32, I32P,
                                 C.POINTER(C.c_int), I64P, I64P]),
    "csb_get_colours": (C.c_int, [P, I32P, C.POINTER(C.c_int)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CE library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CE CUDA library not found at {path}; build it with "
            "`python -m paper_1603_09133_gb300.build` (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
