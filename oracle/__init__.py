"""CPU oracle of the Gaia AVU-GSR PC-LSQR (plain single-threaded FP64 C).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the CUDA library never imports it.  Every routine follows
the definitions cited in gsr_oracle.c (paper §3 column map, Alg. 1 and Alg. 2
for the two products, §2 preconditioning, Paige & Saunders 1982 LSQR).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

STAT_NAMES = ("istop", "itn", "rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm")

_P = ctypes.c_void_p
_I = ctypes.c_int64
_D = ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sysargs = [_I, _I, _I, _P, _P, _P, _P]
        L.or_n_unknowns.argtypes = [_I, _I, _I]
        L.or_n_unknowns.restype = _I
        L.or_aprod1.argtypes = sysargs + [_P, _P]
        L.or_aprod2.argtypes = sysargs + [_P, _P]
        L.or_aprod1_f32.argtypes = sysargs + [_P, _P]
        L.or_aprod2_f32.argtypes = sysargs + [_P, _P]
        L.or_colnorms.argtypes = sysargs + [_P]
        L.or_precondition.argtypes = sysargs + [_P, _P]
        L.or_lsqr.argtypes = sysargs + [_P, _I, _D, _D, _D, _P, _P, _P, _P, ctypes.c_int]
        L.or_lsqr.restype = ctypes.c_int
        L.or_pc_lsqr.argtypes = sysargs + [_P, _I, _D, _D, _D, _P, _P, _P, _P, _P, ctypes.c_int]
        L.or_pc_lsqr.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _sysargs(sys, values=None):
    sp = np.ascontiguousarray(sys.star_ptr, dtype=np.uint32)
    ao = np.ascontiguousarray(sys.attoff, dtype=np.uint32)
    ins = np.ascontiguousarray(sys.instr, dtype=np.uint16)
    val = np.ascontiguousarray(sys.values if values is None else values, dtype=np.float64)
    keep = (sp, ao, ins, val)
    return keep, [sys.n_stars, sys.n_dfa, sys.n_instr, _ptr(sp), _ptr(ao), _ptr(ins), _ptr(val)]


def aprod1(sys, x, y=None, values=None):
    """y += A x (returns y; y defaults to zeros)."""
    keep, a = _sysargs(sys, values)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(sys.m) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().or_aprod1(*a, _ptr(x), _ptr(y))
    return y


def aprod2(sys, y, x=None, values=None):
    """x += A^T y (returns x; x defaults to zeros)."""
    keep, a = _sysargs(sys, values)
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.zeros(sys.n) if x is None else np.array(x, dtype=np.float64, copy=True)
    lib().or_aprod2(*a, _ptr(y), _ptr(x))
    return x


def aprod1_f32(sys, x, y=None):
    """y += A32 x32: binary32 values, vector entries and products, summed in double."""
    keep, a = _sysargs(sys)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(sys.m) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().or_aprod1_f32(*a, _ptr(x), _ptr(y))
    return y


def aprod2_f32(sys, y, x=None):
    """x += A32^T y32: binary32 values, vector entries and products, summed in double."""
    keep, a = _sysargs(sys)
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.zeros(sys.n) if x is None else np.array(x, dtype=np.float64, copy=True)
    lib().or_aprod2_f32(*a, _ptr(y), _ptr(x))
    return x


def colnorms(sys):
    keep, a = _sysargs(sys)
    out = np.empty(sys.n)
    lib().or_colnorms(*a, _ptr(out))
    return out


def precondition(sys):
    """(p, scaled values) with p_j = 1/||A(:,j)|| and scaled = A diag(p)."""
    keep, a = _sysargs(sys)
    p = np.empty(sys.n)
    scaled = np.empty((sys.m, 24))
    lib().or_precondition(*a, _ptr(p), _ptr(scaled))
    return p, scaled


def lsqr(sys, b, itmax, atol=1e-12, btol=1e-12, conlim=1e8, values=None, trace=False,
         run_to_itmax=False):
    """Plain LSQR on the given values (no preconditioning). Returns dict.
    run_to_itmax: iterate to itmax whatever the stopping rules say (they are
    reported for the last iteration)."""
    keep, a = _sysargs(sys, values)
    b = np.ascontiguousarray(b, dtype=np.float64)
    z = np.empty(sys.n)
    var = np.empty(sys.n)
    st = np.zeros(8)
    tr = np.full(max(int(itmax), 1), np.nan) if trace else None
    rc = lib().or_lsqr(*a, _ptr(b), int(itmax), atol, btol, conlim, _ptr(z), _ptr(var), _ptr(st),
                       _ptr(tr) if trace else None, 1 if run_to_itmax else 0)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out = {"z": z, "var": var, **{k: st[i] for i, k in enumerate(STAT_NAMES)}}
    out["istop"], out["itn"] = int(out["istop"]), int(out["itn"])
    if trace:
        out["trace_rnorm"] = tr[: out["itn"]]
    return out


def pc_lsqr(sys, b, itmax, atol=1e-12, btol=1e-12, conlim=1e8, trace=False, run_to_itmax=False):
    """Preconditioned LSQR of the flowchart: returns x, se, p and the stopping
    estimates.  run_to_itmax: iterate to itmax whatever the stopping rules say
    (they are reported for the last iteration)."""
    keep, a = _sysargs(sys)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(sys.n)
    se = np.empty(sys.n)
    p = np.empty(sys.n)
    st = np.zeros(8)
    tr = np.full(max(int(itmax), 1), np.nan) if trace else None
    rc = lib().or_pc_lsqr(*a, _ptr(b), int(itmax), atol, btol, conlim, _ptr(x), _ptr(se), _ptr(p),
                          _ptr(st), _ptr(tr) if trace else None, 1 if run_to_itmax else 0)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out = {"x": x, "se": se, "p": p, **{k: st[i] for i, k in enumerate(STAT_NAMES)}}
    out["istop"], out["itn"] = int(out["istop"]), int(out["itn"])
    if trace:
        out["trace_rnorm"] = tr[: out["itn"]]
    return out


_omp = None


def _omp_lib():
    global _omp
    if _omp is None:
        _build.build()
        L = ctypes.CDLL(_build.OMP_LIB)
        L.cpu_omp_pc_lsqr.argtypes = [_I, _I, _I, _P, _P, _P, _P, _P, _I, _D, _D, _D, _P, _P, _P]
        L.cpu_omp_pc_lsqr.restype = ctypes.c_int
        L.cpu_omp_threads.restype = ctypes.c_int
        _omp = L
    return _omp


def omp_threads() -> int:
    """Threads the OpenMP CPU baseline runs on."""
    return int(_omp_lib().cpu_omp_threads())


def omp_pc_lsqr(sys, b, itmax, atol=1e-12, btol=1e-12, conlim=1e8):
    """The multi-threaded CPU baseline (not the oracle): PC-LSQR as pc_lsqr."""
    keep, a = _sysargs(sys)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(sys.n)
    se = np.empty(sys.n)
    st = np.zeros(8)
    if _omp_lib().cpu_omp_pc_lsqr(*a, _ptr(b), int(itmax), float(atol), float(btol), float(conlim),
                                 _ptr(x), _ptr(se), _ptr(st)) != 0:
        raise MemoryError("cpu_omp_pc_lsqr: allocation failed")
    out = dict(zip(STAT_NAMES, st))
    out["istop"], out["itn"] = int(out["istop"]), int(out["itn"])
    out.update(x=x, se=se)
    return out
