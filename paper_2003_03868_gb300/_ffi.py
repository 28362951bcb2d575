"""ctypes declarations of the C ABI in include/dbcsr_gb.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdbcsr_gb.so")

DBCSR_OK, DBCSR_EINVAL, DBCSR_ENOMEM, DBCSR_ECAPACITY, DBCSR_ECUDA = 0, 1, 2, 3, 4
DBCSR_ENAN, DBCSR_ENOTCONV, DBCSR_ETIMEOUT, DBCSR_ESTATE = 5, 6, 7, 8
DBCSR_FP64, DBCSR_BF16, DBCSR_MIXED, DBCSR_BF16X3, DBCSR_TF32, DBCSR_TF32X3 = 0, 2, 3, 4, 5, 6
DBCSR_PURIFY_TC2, DBCSR_PURIFY_TRS4 = 1, 2
DBCSR_SIGN_FULL_PRODUCTS, DBCSR_SIGN_PLAIN_BF16, DBCSR_SIGN_LOW_CORRECTION, DBCSR_SIGN_RETURN_X = 1, 2, 4, 8
MAX_HISTORY = 128

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECAPACITY", 4: "ECUDA", 5: "ENAN", 6: "ENOTCONV",
                7: "ETIMEOUT", 8: "ESTATE"}


class MultStats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_formed", C.c_int64), ("n_kept", C.c_int64),
                ("n_products", C.c_int64), ("flops", C.c_double), ("dev2_filtered", C.c_double),
                ("ms_symbolic", C.c_double), ("ms_numeric", C.c_double), ("ms_filter", C.c_double),
                ("bytes_min", C.c_double), ("n_launches", C.c_int32), ("reserved", C.c_int32),
                ("flops_tensor", C.c_double), ("bytes_tensor", C.c_double), ("n_tiles", C.c_int64)]


class SignOpts(C.Structure):
    _fields_ = [("eps_filter", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int32), ("prec", C.c_int32),
                ("switch_tol", C.c_double), ("stall_ratio", C.c_double), ("verbose", C.c_int32),
                ("flags", C.c_int32), ("order", C.c_int32), ("reserved", C.c_int32)]


class SignReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("stalled", C.c_int32), ("fp64_from", C.c_int32),
                ("alpha", C.c_double), ("residual", C.c_double), ("trace_p", C.c_double), ("e_band", C.c_double),
                ("flops", C.c_double), ("n_products", C.c_int64), ("ms_total", C.c_double),
                ("ms_multiply", C.c_double), ("nnzb_x", C.c_int64),
                ("residual_history", C.c_double * MAX_HISTORY), ("nnzb_history", C.c_int64 * MAX_HISTORY),
                ("ms_symbolic", C.c_double), ("ms_filter", C.c_double), ("ms_low", C.c_double),
                ("flops_low", C.c_double), ("bytes_min_fp64", C.c_double), ("launches_fp64", C.c_int64),
                ("flops_tensor", C.c_double), ("bytes_tensor", C.c_double)]


class KernelCfg(C.Structure):
    _fields_ = [("tpb", C.c_int32), ("ctas_per_sm", C.c_int32), ("colmajor", C.c_int32), ("prefetch2", C.c_int32),
                ("split", C.c_int32)]


class TuneRecord(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("k", C.c_int32), ("prec", C.c_int32), ("cfg", KernelCfg),
                ("ms", C.c_double), ("gflops", C.c_double)]


class MlpOpts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("reserved", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double)]


class MlpReport(C.Structure):
    _fields_ = [("loss_first", C.c_float), ("loss_last", C.c_float), ("ms", C.c_double), ("epochs", C.c_int32),
                ("reserved", C.c_int32)]


MLP_FEATURES = 12

# (name, restype, argtypes) of every exported entry point
P = C.c_void_p
SIGNATURES = [
    ("dbcsr_last_error", C.c_char_p, []),
    ("dbcsr_version", C.c_char_p, []),
    ("dbcsr_pool_trim", C.c_int, [C.c_uint64]),
    ("dbcsr_multiply_plan", C.c_int, [C.c_double, P, P, P, C.c_double, C.c_int32, C.POINTER(P),
                                      C.POINTER(MultStats)]),
    ("dbcsr_multiply_execute", C.c_int, [P]),
    ("dbcsr_plan_destroy", C.c_int, [P]),
    ("dbcsr_put_values", C.c_int, [P, P, C.c_int]),
    ("dbcsr_tune_predicted", C.c_int, [C.c_int32, P, P, C.c_int32, C.c_int64, C.c_int32, C.c_double, P]),
    ("dbcsr_create", C.c_int, [C.POINTER(P), C.c_int32, P, P]),
    ("dbcsr_destroy", C.c_int, [P]),
    ("dbcsr_put_block", C.c_int, [P, C.c_int32, C.c_int32, P, C.c_int]),
    ("dbcsr_put_blocks", C.c_int, [P, C.c_int64, P, P, P, C.c_int]),
    ("dbcsr_finalize", C.c_int, [P]),
    ("dbcsr_get_info", C.c_int, [P, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("dbcsr_get_block", C.c_int, [P, C.c_int32, C.c_int32, P, C.POINTER(C.c_int)]),
    ("dbcsr_export", C.c_int, [P, P, P, P]),
    ("dbcsr_copy", C.c_int, [P, P]),
    ("dbcsr_scale_shift", C.c_int, [P, C.c_double, C.c_double]),
    ("dbcsr_multiply", C.c_int, [C.c_double, P, P, C.c_double, P, C.c_double, C.c_int32, C.POINTER(MultStats)]),
    ("dbcsr_add", C.c_int, [C.c_double, P, C.c_double, P]),
    ("dbcsr_save", C.c_int, [P, C.c_char_p]),
    ("dbcsr_load", C.c_int, [C.POINTER(P), C.c_char_p, P]),
    ("dbcsr_file_info", C.c_int, [C.c_char_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("dbcsr_filter", C.c_int, [P, C.c_double]),
    ("dbcsr_trace", C.c_int, [P, C.POINTER(C.c_double)]),
    ("dbcsr_trace_product", C.c_int, [P, P, C.POINTER(C.c_double)]),
    ("dbcsr_trace_product_noalloc", C.c_int, [P, P, P]),
    ("dbcsr_gershgorin", C.c_int, [P, C.c_double, C.POINTER(C.c_double)]),
    ("dbcsr_sign_iterate", C.c_int, [P, C.c_double, C.POINTER(SignOpts), P, C.POINTER(SignReport)]),
    ("dbcsr_sign_iterate_resume", C.c_int, [P, P, C.POINTER(SignReport), C.POINTER(SignOpts), P,
                                            C.POINTER(SignReport)]),
    ("dbcsr_inverse_hotelling", C.c_int, [P, C.POINTER(SignOpts), P, C.POINTER(SignReport)]),
    ("dbcsr_inverse_sqrt", C.c_int, [P, C.POINTER(SignOpts), P, P, C.POINTER(SignReport)]),
    ("dbcsr_submatrix_sign", C.c_int, [P, C.c_double, C.POINTER(SignOpts), P, C.POINTER(SignReport)]),
    ("dbcsr_purify", C.c_int, [P, C.c_double, C.c_int32, C.POINTER(SignOpts), P, C.POINTER(SignReport)]),
    ("dbcsr_sign_mu_search", C.c_int, [P, C.c_double, C.c_double, C.c_double, C.POINTER(SignOpts), P,
                                       C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(SignReport)]),
    ("dbcsr_sign_iterate_nonorth", C.c_int, [P, P, C.c_double, C.POINTER(SignOpts), P, C.POINTER(SignReport),
                                             C.POINTER(SignReport)]),
    ("dbcsr_sign_iterate_batched", C.c_int, [C.c_int32, P, P, C.POINTER(SignOpts), P, P]),
    ("dbcsr_tune_space", C.c_int, [C.c_int32, P, C.c_int32, C.POINTER(C.c_int32)]),
    ("dbcsr_autotune", C.c_int, [P, C.c_int32, C.c_int32, C.c_int64, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    ("dbcsr_time_config", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int32, P, C.c_int32, P]),
    ("dbcsr_tune_set", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, P]),
    ("dbcsr_tune_get", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, C.POINTER(C.c_int)]),
    ("dbcsr_tune_clear", C.c_int, []),
    ("dbcsr_tune_save", C.c_int, [C.c_char_p]),
    ("dbcsr_tune_load", C.c_int, [C.c_char_p]),
    ("dbcsr_mlp_param_count", C.c_int64, [C.c_int32]),
    ("dbcsr_mlp_init", C.c_int, [C.c_int32, C.c_uint64, P]),
    ("dbcsr_mlp_features", C.c_int, [C.c_int32, P, P, C.c_int64, P]),
    ("dbcsr_mlp_forward", C.c_int, [C.c_int32, P, P, C.c_int64, P]),
    ("dbcsr_mlp_loss_grad", C.c_int, [C.c_int32, P, P, P, C.c_int64, C.POINTER(C.c_float), P]),
    ("dbcsr_mlp_train", C.c_int, [C.c_int32, P, P, P, C.c_int64, C.POINTER(MlpOpts), C.POINTER(MlpReport)]),
    ("dbcsr_mlp_predict_best", C.c_int, [C.c_int32, P, P, C.c_int32, P, P]),
    ("dbcsr_tune_records_save", C.c_int, [C.c_char_p, P, C.c_int64, C.c_int32]),
    ("dbcsr_predictor_train", C.c_int, [C.c_char_p, C.c_int32, C.c_uint64, C.POINTER(MlpOpts), C.POINTER(MlpReport)]),
    ("dbcsr_predictor_data", C.c_int, [C.c_char_p, C.c_int32, P, P, C.c_int64, C.POINTER(C.c_int64)]),
    ("dbcsr_predictor_params", C.c_int, [C.c_int32, P]),
    ("dbcsr_partition_rows", C.c_int, [C.c_int32, P, P, C.c_int32, P]),
    ("dbcsr_set_fp64_schedule", C.c_int, [C.c_int32]),
    ("dbcsr_dense_multiply", C.c_int, [C.c_int32, C.c_int64, C.c_int32, C.c_double, P, P, C.c_double, P, P]),
    ("dbcsr_get_fp64_schedule", C.c_int32, []),
    ("dbcsr_halo_rows", C.c_int, [C.c_int32, P, P, P, C.c_int32, P, C.c_int32, C.POINTER(C.c_int32)]),
    ("dbcsr_bench_peak", C.c_double, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    ("dbcsr_launch_count", C.c_int64, []),
    ("dbcsr_pool_usage", C.c_int32, [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32]),
    ("dbcsr_wait_selftest", C.c_int32, [C.c_int64, C.c_int32, C.POINTER(C.c_int64)]),
    ("dbcsr_matrix_groups", C.c_int32, [P, P, P, C.POINTER(C.c_int32)]),
]

_lib = None


def load():
    """The shared library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2003_03868_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
