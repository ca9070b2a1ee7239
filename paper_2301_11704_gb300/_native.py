"""ctypes binding of libksconn.so (include/ksconn.h): argument marshalling only.

Every computation runs in the CUDA library.  Loading fails loudly when the
library has not been built (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

KS_OK, KS_EINVAL, KS_ENOMEM, KS_ECUDA, KS_ETIMEOUT, KS_ENONFINITE, KS_ENOTCONV, KS_ENOTEQUILIBRIUM, KS_ENOTIMPL = range(9)
STATUS_NAMES = {0: "KS_OK", 1: "KS_EINVAL", 2: "KS_ENOMEM", 3: "KS_ECUDA", 4: "KS_ETIMEOUT",
                5: "KS_ENONFINITE", 6: "KS_ENOTCONV", 7: "KS_ENOTEQUILIBRIUM", 8: "KS_ENOTIMPL"}
KS_FP64, KS_FP32, KS_BF16X2, KS_BF16X3 = 0, 1, 2, 3
KS_ADJ_PAPER, KS_ADJ_DISCRETE = 0, 1
KS_CONV_JARC, KS_CONV_J, KS_CONV_JREL = 0, 1, 2
KS_SCHEME_IMEX, KS_SCHEME_IMPLICIT = 0, 1
KS_SYM_ODD, KS_SYM_HALF_PERIOD, KS_SYM_SINE = 1, 2, 4

# Every symbol include/ksconn.h declares.
EXPORTS = [
    "ks_last_error", "ks_version", "ks_curve_workspace_bytes", "ks_curve_fft_length", "ks_curve_s_form", "ks_curve_create", "ks_curve_set_stream",
    "ks_curve_init_trial", "ks_curve_residual", "ks_curve_cost", "ks_curve_gradient", "ks_curve_descend",
    "ks_curve_descend_async", "ks_curve_scalars", "ks_curve_get_state", "ks_curve_set_state", "ks_curve_profile",
    "ks_curve_profile_read", "ks_curve_debug_wait_limit", "ks_curve_destroy", "ks_cost_noalloc",
    "ks_batch_workspace_bytes", "ks_batch_create", "ks_batch_init_trial", "ks_batch_descend",
    "ks_batch_descend_async", "ks_batch_scalars", "ks_batch_get_state", "ks_batch_autotune", "ks_batch_get_tuning",
    "ks_batch_destroy",
]


class KSParams(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("nx", ctypes.c_int32),
        ("ns", ctypes.c_int32),
        ("S", ctypes.c_double),
        ("s0", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("lambda_free", ctypes.c_int32),
        ("dtau", ctypes.c_double),
        ("dtau_lambda", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("adjoint", ctypes.c_int32),
        ("conv", ctypes.c_int32),
        ("check_ends", ctypes.c_int32),
        ("symmetry", ctypes.c_int32),
        ("s_transform", ctypes.c_int32),
        ("launch", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
    ]


class KSScalars(ctypes.Structure):
    _fields_ = [
        ("J", ctypes.c_double),
        ("J_arc", ctypes.c_double),
        ("dJ2_dlambda", ctypes.c_double),
        ("G_norm", ctypes.c_double),
        ("Dnorm", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("step", ctypes.c_int64),
        ("converged", ctypes.c_int32),
        ("status", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KSProfile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 3), ("launches", ctypes.c_int64 * 3), ("step_ms", ctypes.c_double),
                ("step_launches", ctypes.c_int64), ("step_steps", ctypes.c_int64),
                ("pass_ms", (ctypes.c_double * 3) * 2), ("pass_launches", (ctypes.c_int64 * 3) * 2),
                ("impl_ms", ctypes.c_double), ("impl_launches", ctypes.c_int64)]


class KSBatchTuning(ctypes.Structure):
    _fields_ = [("row_sections", ctypes.c_int32), ("dense_tile", ctypes.c_int32), ("nlen", ctypes.c_int32),
                ("F", ctypes.c_int32 * 8), ("F1", ctypes.c_int32 * 8), ("ms_per_step", ctypes.c_double)]


class KSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libksconn.so (building it with nvcc first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libksconn.so is not built (%s); run paper_2301_11704_gb300.build.build()" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    p, i32, i64, d, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    pd, pi64 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    sigs = {
        "ks_last_error": (ctypes.c_char_p, []),
        "ks_version": (i32, []),
        "ks_curve_workspace_bytes": (sz, [ctypes.POINTER(KSParams)]),
        "ks_curve_fft_length": (i32, [ctypes.POINTER(KSParams)]),
        "ks_curve_s_form": (i32, [ctypes.POINTER(KSParams)]),
        "ks_curve_create": (i32, [ctypes.POINTER(KSParams), pd, pd, p, p, sz, p, ctypes.POINTER(p)]),
        "ks_curve_set_stream": (i32, [p, p]),
        "ks_curve_init_trial": (i32, [p, d, pd, i32, pd, pd]),
        "ks_curve_residual": (i32, [p, p]),
        "ks_curve_cost": (i32, [p, pd, pd]),
        "ks_curve_gradient": (i32, [p, i32, p, pd]),
        "ks_curve_descend": (i32, [p, i64, d, pi64, pd, pd]),
        "ks_curve_descend_async": (i32, [p, i64, d]),
        "ks_curve_scalars": (i32, [p, ctypes.POINTER(KSScalars)]),
        "ks_curve_get_state": (i32, [p, p, pd, pd]),
        "ks_curve_set_state": (i32, [p, p, d, d]),
        "ks_curve_profile": (i32, [p, i32]),
        "ks_curve_profile_read": (i32, [p, ctypes.POINTER(KSProfile)]),
        "ks_curve_debug_wait_limit": (i32, [p, i64]),
        "ks_curve_destroy": (i32, [p]),
        "ks_cost_noalloc": (i32, [ctypes.POINTER(KSParams), p, p, p]),
        "ks_batch_workspace_bytes": (sz, [i32, ctypes.POINTER(KSParams)]),
        "ks_batch_create": (i32, [i32, ctypes.POINTER(KSParams), pd, pd, p, sz, p, ctypes.POINTER(p)]),
        "ks_batch_init_trial": (i32, [p, i32, pd, pd]),
        "ks_batch_descend": (i32, [p, i64, d, pi64, pd, pd]),
        "ks_batch_descend_async": (i32, [p, i64, d]),
        "ks_batch_scalars": (i32, [p, ctypes.POINTER(KSScalars)]),
        "ks_batch_get_state": (i32, [p, i32, p]),
        "ks_batch_autotune": (i32, [p, i32, ctypes.POINTER(i32)]),
        "ks_batch_get_tuning": (i32, [p, ctypes.POINTER(KSBatchTuning)]),
        "ks_batch_destroy": (i32, [p]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, allow=()) -> int:
    if status != KS_OK and status not in allow:
        msg = _lib.ks_last_error().decode(errors="replace") if _lib is not None else ""
        raise KSError(status, msg)
    return status


def dptr(arr):
    """Pointer to a contiguous float64 numpy array (or None)."""
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
