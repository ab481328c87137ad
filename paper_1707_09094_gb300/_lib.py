"""ctypes binding of the C ABI in include/gmm_gb300.h (argument marshalling only).

Each ``gmm_*`` function here has the C function's name and arguments; every
step of the computation runs in the CUDA library.  Loading fails loudly when
the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgmm_gb300.so")

GMM_OK, GMM_ERR_ARG, GMM_ERR_NONFINITE, GMM_ERR_CUDA = 0, -1, -2, -3
GMM_ERR_TIMEOUT, GMM_ERR_OOM, GMM_ERR_STATE, GMM_ERR_UNSUPPORTED = -4, -5, -6, -7
GMM_EUCL, GMM_MAHA, GMM_PROB = 0, 1, 2
GMM_KEEP_EXISTING, GMM_RANDOM_SUBSET, GMM_STATIC_SUBSET, GMM_STATIC_SPREAD, GMM_RANDOM_SPREAD = 0, 1, 2, 3, 4
GMM_FP32, GMM_BF16 = 0, 1
GMM_DEBUG_WAIT_CYCLES, GMM_DEBUG_SKIP_MMA, GMM_DEBUG_KM_FORM, GMM_DEBUG_FP32_FORM, GMM_DEBUG_TC_FORM = 1, 2, 3, 4, 5
GMM_STAT_SCREENED, GMM_STAT_KEPT, GMM_STAT_DENSE = 3, 4, 5
GMM_STAT_KM_SCREENED, GMM_STAT_KM_DEFERRED, GMM_STAT_KM_FP64 = 14, 15, 16

STATUS_NAMES = {0: "GMM_OK", -1: "GMM_ERR_ARG", -2: "GMM_ERR_NONFINITE", -3: "GMM_ERR_CUDA",
                -4: "GMM_ERR_TIMEOUT", -5: "GMM_ERR_OOM", -6: "GMM_ERR_STATE", -7: "GMM_ERR_UNSUPPORTED"}


class gmm_learn_opts(ctypes.Structure):
    _fields_ = [("dist", ctypes.c_int32), ("seed_mode", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("em_tol", ctypes.c_double), ("prec", ctypes.c_int32), ("print", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


P = ctypes.c_void_p
i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "gmm_create": (ctypes.c_int, [ctypes.POINTER(P)]),
    "gmm_destroy": (None, [P]),
    "gmm_default_opts": (None, [ctypes.POINTER(gmm_learn_opts)]),
    "gmm_learn": (ctypes.c_int, [P, P, i64, i32, i32, i32, i32, f64, ctypes.POINTER(gmm_learn_opts)]),
    "gmm_em_iterate": (ctypes.c_int, [P, P, i64, i32, f64, i32, i32, P]),
    "gmm_learn_batched": (ctypes.c_int, [P, i32, P, P, P, P, i32, i32, f64, ctypes.POINTER(gmm_learn_opts)]),
    "gmm_kmeans": (ctypes.c_int, [P, P, i64, i32, i32, f64, P, P]),
    "gmm_log_p": (ctypes.c_int, [P, P, i64, i32, P, P]),
    "gmm_avg_log_p": (ctypes.c_int, [P, P, i64, i32, ctypes.POINTER(f64), P]),
    "gmm_avg_log_p_noalloc": (ctypes.c_int, [P, P, i64, i32, ctypes.POINTER(f64), P]),
    "gmm_assign": (ctypes.c_int, [P, P, i64, i32, P, P]),
    "gmm_raw_hist": (ctypes.c_int, [P, P, i64, i32, P, P]),
    "gmm_norm_hist": (ctypes.c_int, [P, P, i64, i32, P, P]),
    "gmm_get_params": (ctypes.c_int, [P, ctypes.POINTER(i32), ctypes.POINTER(i32), P, P, P]),
    "gmm_set_params": (ctypes.c_int, [P, i32, i32, P, P, P]),
    "gmm_generate": (ctypes.c_int, [P, i64, ctypes.c_uint64, P, P]),
    "gmm_x_from_f64": (ctypes.c_int, [P, i64, P, P]),
    "gmm_save": (ctypes.c_int, [P, ctypes.c_char_p]),
    "gmm_load": (ctypes.c_int, [P, ctypes.c_char_p]),
    "gmm_get_stats": (ctypes.c_int, [P, P, i32, ctypes.POINTER(i32)]),
    "gmm_profile": (ctypes.c_int, [P, i32]),
    "gmm_profile_read": (ctypes.c_int, [P, ctypes.POINTER(f64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "gmm_debug_set": (ctypes.c_int, [P, i32, i64]),
    "gmm_debug_get": (ctypes.c_int, [P, i32, ctypes.POINTER(i64)]),
    "gmm_init_net_create": (ctypes.c_int, [ctypes.POINTER(P), i32, i32, i32, i32, i32, i32, ctypes.c_uint64]),
    "gmm_init_net_destroy": (None, [P]),
    "gmm_init_net_num_params": (i64, [P]),
    "gmm_init_net_get_weights": (ctypes.c_int, [P, P, P]),
    "gmm_init_net_set_weights": (ctypes.c_int, [P, P]),
    "gmm_init_net_get_adam": (ctypes.c_int, [P, P, P, P]),
    "gmm_init_net_set_adam": (ctypes.c_int, [P, P, P, i64]),
    "gmm_init_net_step": (ctypes.c_int, [P, P, i32, i32, P, P, P, f64, f64, i32, f64, P, P, P,
                                         ctypes.POINTER(f64), P]),
    "gmm_init_net_seed_model": (ctypes.c_int, [P, P, P, i64, i32, ctypes.c_uint64, f64, P]),
    "gmm_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load the built library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is not built; run paper_1707_09094_gb300.build.build() "
                               "(there is no CPU fallback)" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GmmError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().gmm_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status: int, where: str):
    if status != GMM_OK:
        raise GmmError(status, where)


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
