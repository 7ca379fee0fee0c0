"""ctypes view of libgsr.so (the C ABI declared in include/gsr.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library cannot be built or loaded;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

GSR_OK = 0
GSR_ERR_ARG = -1
GSR_ERR_INDEX = -2
GSR_ERR_OOM = -3
GSR_ERR_CUDA = -4
GSR_ERR_TIMEOUT = -5
GSR_ERR_NONFINITE = -6
GSR_ERR_UNSUPPORTED = -7

GSR_PREC_FP64 = 0
GSR_PREC_MIXED = 1
GSR_INSTR_AUTO, GSR_INSTR_SMEM, GSR_INSTR_REPLICAS, GSR_INSTR_SORTED = 0, 1, 2, 3
GSR_PRODUCTS_AUTO, GSR_PRODUCTS_NATIVE, GSR_PRODUCTS_SPLIT = 0, 1, 2
GSR_PRODUCTS_MASK = 0x100
GSR_SPLIT_APROD1, GSR_SPLIT_APROD2_STARS, GSR_SPLIT_APROD2_INSTR = 1, 2, 4
GSR_SPLIT_APROD2_ATT, GSR_SPLIT_APROD2_ATT2, GSR_SPLIT_APROD1_ASTRO = 8, 16, 32

EXPORTS = (
    "gsr_config_default", "gsr_create", "gsr_destroy", "gsr_aprod1", "gsr_aprod2",
    "gsr_precondition", "gsr_lsqr_solve", "gsr_last_error", "gsr_info", "gsr_strerror",
    "gsr_aprod1_norm_noalloc", "gsr_aprod1_f32", "gsr_aprod2_f32", "gsr_mixed_solve",
    "gsr_set_values", "gsr_normal_solve", "gsr_lsq_backward", "gsr_batched_solve",
    "gsr_batched_products", "gsr_set_batch_tiling", "gsr_set_aprod2_fused",
    "gsr_product_forms", "gsr_fp64_fma_rate", "gsr_time_iteration", "gsr_vector_add",
    "gsr_set_aprod1_staging", "gsr_aprod1_staging", "gsr_kernel_status",
    "gsr_inject_missing_copy",
)


class Dims(ctypes.Structure):
    _fields_ = [("n_stars", ctypes.c_int64), ("n_dfa", ctypes.c_int64),
                ("n_instr", ctypes.c_int64), ("n_rows", ctypes.c_int64)]


class Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("conlim", ctypes.c_double),
                ("lanes_per_star", ctypes.c_int), ("validate", ctypes.c_int),
                ("force_itmax", ctypes.c_int), ("eager", ctypes.c_int),
                ("instr_mode", ctypes.c_int), ("products", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("istop", ctypes.c_int), ("itn", ctypes.c_int), ("rnorm", ctypes.c_double),
                ("arnorm", ctypes.c_double), ("anorm", ctypes.c_double),
                ("acond", ctypes.c_double), ("xnorm", ctypes.c_double),
                ("bnorm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MixedResult(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer", ctypes.c_int), ("inner", ctypes.c_int),
                ("rnorm", ctypes.c_double), ("arnorm", ctypes.c_double),
                ("anorm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CgResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_resid", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GsrError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = lib()
        msg = L.gsr_strerror(code).decode()
        detail = L.gsr_last_error().decode()
        super().__init__("%s: %s (%d)%s" % (where, msg, code, (": " + detail) if detail else ""))
        self.code = code


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libgsr.so is missing and could not be built")
            L = ctypes.CDLL(path)
            P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            L.gsr_config_default.argtypes = [ctypes.POINTER(Config)]
            L.gsr_config_default.restype = None
            L.gsr_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Dims), P, P, P, P,
                                     ctypes.POINTER(Config)]
            L.gsr_destroy.argtypes = [P]
            L.gsr_aprod1.argtypes = [P, P, P, P]
            L.gsr_aprod2.argtypes = [P, P, P, P]
            L.gsr_precondition.argtypes = [P, P, P]
            L.gsr_lsqr_solve.argtypes = [P, P, I, D, D, P, P, ctypes.POINTER(Result), P]
            L.gsr_aprod1_norm_noalloc.argtypes = [P, P, P, D, P, P]
            L.gsr_aprod1_f32.argtypes = [P, P, P, P]
            L.gsr_aprod2_f32.argtypes = [P, P, P, P]
            L.gsr_mixed_solve.argtypes = [P, P, I, I, D, D, P, ctypes.POINTER(MixedResult), P]
            L.gsr_set_values.argtypes = [P, I, P, P]
            L.gsr_normal_solve.argtypes = [P, P, I, D, P, ctypes.POINTER(CgResult), P]
            L.gsr_lsq_backward.argtypes = [P, P, P, P, I, D, P, P, ctypes.POINTER(CgResult), P]
            L.gsr_batched_solve.argtypes = [P, I, P, I, I, D, D, P, ctypes.POINTER(MixedResult), P]
            L.gsr_batched_products.argtypes = [P, I, P, P, P, P, P]
            L.gsr_set_batch_tiling.argtypes = [P, I, I]
            L.gsr_set_aprod2_fused.argtypes = [P, I]
            L.gsr_product_forms.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
            L.gsr_fp64_fma_rate.argtypes = [ctypes.POINTER(D)]
            L.gsr_time_iteration.argtypes = [P, P, I, P, P]
            L.gsr_vector_add.argtypes = [P, P, I64, P]
            L.gsr_set_aprod1_staging.argtypes = [P, I]
            L.gsr_aprod1_staging.argtypes = [P, ctypes.POINTER(I)]
            L.gsr_kernel_status.argtypes = [P, P]
            L.gsr_inject_missing_copy.argtypes = [P, I64]
            L.gsr_last_error.restype = ctypes.c_char_p
            L.gsr_strerror.argtypes = [I]
            L.gsr_strerror.restype = ctypes.c_char_p
            L.gsr_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
            for name in ("gsr_create", "gsr_destroy", "gsr_aprod1", "gsr_aprod2",
                         "gsr_precondition", "gsr_lsqr_solve", "gsr_info",
                         "gsr_aprod1_norm_noalloc", "gsr_aprod1_f32", "gsr_aprod2_f32",
                         "gsr_mixed_solve", "gsr_set_values", "gsr_normal_solve",
                         "gsr_lsq_backward", "gsr_batched_solve", "gsr_batched_products",
                         "gsr_set_batch_tiling", "gsr_set_aprod2_fused", "gsr_product_forms",
                         "gsr_fp64_fma_rate", "gsr_time_iteration", "gsr_vector_add",
                         "gsr_set_aprod1_staging", "gsr_aprod1_staging", "gsr_kernel_status",
                         "gsr_inject_missing_copy"):
                getattr(L, name).restype = I
            _lib = L
    return _lib


def check(code: int, where: str) -> None:
    if code != GSR_OK:
        raise GsrError(code, where)
