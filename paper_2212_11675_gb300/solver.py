"""Python face of the C ABI: a Solver owning one gsr handle.

Vectors may be CUDA tensors (device pointers are passed straight through) or
NumPy arrays (host pointers: the library stages them through device memory
inside the call).  PyTorch only provides device memory and streams here.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import CgResult, Config, Dims, MixedResult, Result, check, lib


def _torch():
    import torch
    return torch


def _ptr(a):
    """(pointer, keepalive) of a CUDA tensor or a host NumPy array."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _check_vec(a, n, name, dtype=np.float64):
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or a.size != n:
            raise ValueError("%s must be %s[%d]" % (name, np.dtype(dtype).name, n))
    else:
        torch = _torch()
        want = {np.float64: torch.float64}[dtype]
        if a.dtype != want or a.numel() != n:
            raise ValueError("%s must be %s[%d]" % (name, want, n))


def _stream(stream):
    if stream is None:
        try:
            torch = _torch()
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Solver:
    """PC-LSQR solver of one Gaia observation system (paper §3 structure)."""

    def __init__(self, system, conlim: float = 1e8, lanes_per_star: int = 0,
                 validate: bool = True, precision: int = _lib.GSR_PREC_FP64,
                 force_itmax: bool = False, eager: bool = False, instr_mode: int = 0,
                 products: int = 0):
        L = lib()
        self._h = ctypes.c_void_p()
        d = Dims(system.n_stars, system.n_dfa, system.n_instr, int(system.m))
        cfg = Config()
        L.gsr_config_default(ctypes.byref(cfg))
        cfg.conlim = conlim
        cfg.lanes_per_star = lanes_per_star
        cfg.validate = 1 if validate else 0
        cfg.precision = precision
        cfg.force_itmax = 1 if force_itmax else 0
        cfg.eager = 1 if eager else 0
        cfg.instr_mode = instr_mode
        cfg.products = products
        arrs = []
        for a, dt in ((system.star_ptr, np.uint32), (system.attoff, np.uint32),
                      (system.instr, np.uint16), (system.values, np.float64)):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=dt)
            arrs.append(a)
        ptrs = [_ptr(a)[0] for a in arrs]
        check(L.gsr_create(ctypes.byref(self._h), ctypes.byref(d), *ptrs, ctypes.byref(cfg)),
              "gsr_create")
        self.n_stars, self.n_dfa, self.n_instr = system.n_stars, system.n_dfa, system.n_instr
        m, n, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(L.gsr_info(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(b)), "gsr_info")
        self.m, self.n, self.device_bytes = m.value, n.value, b.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gsr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def aprod1(self, x, y, stream=None):
        """y += A x (paper Alg. 1); returns y."""
        _check_vec(x, self.n, "x")
        _check_vec(y, self.m, "y")
        check(lib().gsr_aprod1(self._h, _ptr(x)[0], _ptr(y)[0], _stream(stream)), "gsr_aprod1")
        return y

    def aprod2(self, y, x, stream=None):
        """x += A^T y (paper Alg. 2); returns x."""
        _check_vec(y, self.m, "y")
        _check_vec(x, self.n, "x")
        check(lib().gsr_aprod2(self._h, _ptr(y)[0], _ptr(x)[0], _stream(stream)), "gsr_aprod2")
        return x

    def aprod1_f32(self, x, y, stream=None):
        """y += A32 x with binary32 products (mixed-precision handles); returns y."""
        _check_vec(x, self.n, "x")
        _check_vec(y, self.m, "y")
        check(lib().gsr_aprod1_f32(self._h, _ptr(x)[0], _ptr(y)[0], _stream(stream)),
              "gsr_aprod1_f32")
        return y

    def aprod2_f32(self, y, x, stream=None):
        """x += A32^T y with binary32 products (mixed-precision handles); returns x."""
        _check_vec(y, self.m, "y")
        _check_vec(x, self.n, "x")
        check(lib().gsr_aprod2_f32(self._h, _ptr(y)[0], _ptr(x)[0], _stream(stream)),
              "gsr_aprod2_f32")
        return x

    def mixed_solve(self, b, max_outer=10, max_inner=100, inner_tol=1e-4, atol=1e-12, x=None,
                    stream=None):
        """Mixed-precision PC least squares (binary32 inner CG, FP64 refinement);
        returns (x, result dict)."""
        _check_vec(b, self.m, "b")
        if x is None:
            x = np.empty(self.n) if isinstance(b, np.ndarray) else _torch().empty(
                self.n, dtype=b.dtype, device=b.device)
        _check_vec(x, self.n, "x")
        res = MixedResult()
        check(lib().gsr_mixed_solve(self._h, _ptr(b)[0], int(max_outer), int(max_inner),
                                    float(inner_tol), float(atol), _ptr(x)[0], ctypes.byref(res),
                                    _stream(stream)), "gsr_mixed_solve")
        return x, res.as_dict()

    def set_values(self, k, values, stream=None):
        """Replace nonzero k (0..23; 23 = global column) of every row."""
        _check_vec(values, self.m, "values")
        check(lib().gsr_set_values(self._h, int(k), _ptr(values)[0], _stream(stream)),
              "gsr_set_values")

    def normal_solve(self, g, max_iter=1000, tol=1e-13, q=None, stream=None):
        """q = (A^T A)^{-1} g by FP64 conjugate gradients; returns (q, info)."""
        _check_vec(g, self.n, "g")
        if q is None:
            q = np.empty(self.n) if isinstance(g, np.ndarray) else _torch().empty_like(g)
        res = CgResult()
        check(lib().gsr_normal_solve(self._h, _ptr(g)[0], int(max_iter), float(tol), _ptr(q)[0],
                                     ctypes.byref(res), _stream(stream)), "gsr_normal_solve")
        return q, res.as_dict()

    def lsq_backward(self, b, x, gx, max_iter=1000, tol=1e-13, want_glob=True, stream=None):
        """(dL/db, dL/dA(:, global), info) for the least-squares solution x of b."""
        _check_vec(b, self.m, "b")
        _check_vec(x, self.n, "x")
        _check_vec(gx, self.n, "gx")
        host = isinstance(b, np.ndarray)
        mk = (lambda: np.empty(self.m)) if host else (
            lambda: _torch().empty(self.m, dtype=b.dtype, device=b.device))
        gb = mk()
        gg = mk() if want_glob else None
        res = CgResult()
        check(lib().gsr_lsq_backward(self._h, _ptr(b)[0], _ptr(x)[0], _ptr(gx)[0], int(max_iter),
                                     float(tol), _ptr(gb)[0], _ptr(gg)[0] if gg is not None else None,
                                     ctypes.byref(res), _stream(stream)), "gsr_lsq_backward")
        return gb, gg, res.as_dict()

    def set_aprod2_fused(self, fused):
        """aprod 2 (sorted instrumental path) in one launch with a shared work
        queue (True, the default) or as separate passes (False)."""
        check(lib().gsr_set_aprod2_fused(self._h, 1 if fused else 0), "gsr_set_aprod2_fused")

    def set_aprod1_staging(self, staged):
        """FP64 aprod 1 with its tiles staged in shared memory by the bulk-copy
        engine (True) or loaded into registers (False); bitwise-equal results."""
        check(lib().gsr_set_aprod1_staging(self._h, 1 if staged else 0),
              "gsr_set_aprod1_staging")

    def aprod1_staging(self):
        v = ctypes.c_int()
        check(lib().gsr_aprod1_staging(self._h, ctypes.byref(v)), "gsr_aprod1_staging")
        return bool(v.value)

    def kernel_status(self, stream=None):
        """Raw status of the bounded device waits since the last check
        (GSR_OK or GSR_ERR_TIMEOUT; the flag is cleared)."""
        return lib().gsr_kernel_status(self._h, _stream(stream))

    def inject_missing_copy(self, tile):
        """Test hook: tile's bulk copies are never issued (-1: off)."""
        check(lib().gsr_inject_missing_copy(self._h, int(tile)), "gsr_inject_missing_copy")

    def product_forms(self):
        """(aprod1_split, aprod2_split): which FP64 products run on the binary32
        pipes from exact splits: aprod1_split 0 (none), 1 (instrumental and
        global) or 2 (also astrometric), aprod2_split a set of bits (1 star
        units, 2 instrument units, 4 and 8 the axis-2 and axes-1-2 taps of the
        attitude units of the single-launch aprod 2)."""
        a1, a2 = ctypes.c_int(), ctypes.c_int()
        check(lib().gsr_product_forms(self._h, ctypes.byref(a1), ctypes.byref(a2)),
              "gsr_product_forms")
        return int(a1.value), int(a2.value)

    def time_iteration(self, b, iters=20, stream=None):
        """Average durations (ms) of aprod 1, aprod 2 and the vector pass of an
        LSQR iteration as they run inside a solve of b (CUDA events)."""
        _check_vec(b, self.m, "b")
        out = np.zeros(3)
        check(lib().gsr_time_iteration(self._h, _ptr(b)[0], int(iters),
                                       out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
              "gsr_time_iteration")
        return {"aprod1": float(out[0]), "aprod2": float(out[1]), "vector_pass": float(out[2])}

    def set_batch_tiling(self, kt, lanes):
        """Column tile (1, 2, 4, 8) and lanes per star (8, 16, 32) of the batched kernels."""
        check(lib().gsr_set_batch_tiling(self._h, int(kt), int(lanes)), "gsr_set_batch_tiling")

    def batched_products(self, X, Y, stream=None):
        """(A32 X, A32^T Y) for X (k, n) and Y (k, m) CUDA tensors (rows are columns)."""
        torch = _torch()
        k = X.shape[0]
        if X.shape != (k, self.n) or Y.shape != (k, self.m):
            raise ValueError("X must be (k, n) and Y (k, m)")
        Q = torch.empty((k, self.m), dtype=torch.float64, device=X.device)
        T = torch.empty((k, self.n), dtype=torch.float64, device=X.device)
        check(lib().gsr_batched_products(self._h, k, _ptr(X)[0], _ptr(Y)[0], _ptr(Q)[0], _ptr(T)[0],
                                         _stream(stream)), "gsr_batched_products")
        return Q, T

    def batched_solve(self, B, max_outer=10, max_inner=100, inner_tol=1e-4, atol=1e-12,
                      stream=None):
        """Mixed-precision least squares for k right-hand sides B (k, m); returns
        (X (k, n), list of k result dicts)."""
        k = B.shape[0]
        if B.shape != (k, self.m):
            raise ValueError("B must be (k, m)")
        if isinstance(B, np.ndarray):
            B = np.ascontiguousarray(B, dtype=np.float64)
            X = np.empty((k, self.n))
        else:
            B = B.contiguous()
            X = _torch().empty((k, self.n), dtype=B.dtype, device=B.device)
        res = (MixedResult * k)()
        check(lib().gsr_batched_solve(self._h, k, _ptr(B)[0], int(max_outer), int(max_inner),
                                      float(inner_tol), float(atol), _ptr(X)[0], res,
                                      _stream(stream)), "gsr_batched_solve")
        return X, [r.as_dict() for r in res]

    def precondition(self, p, stream=None):
        """p = 1/||A(:,j)|| (1 for an empty column); returns p."""
        _check_vec(p, self.n, "p")
        check(lib().gsr_precondition(self._h, _ptr(p)[0], _stream(stream)), "gsr_precondition")
        return p

    def lsqr_solve(self, b, itmax, atol=1e-12, btol=1e-12, x=None, se=None, stream=None,
                   want_se=True):
        """PC-LSQR: returns (x, se, result dict).  Output buffers default to
        arrays on the same side (host or device) as b."""
        _check_vec(b, self.m, "b")
        if x is None:
            x = np.empty(self.n) if isinstance(b, np.ndarray) else _torch().empty(
                self.n, dtype=b.dtype, device=b.device)
        if se is None and want_se:
            se = np.empty(self.n) if isinstance(b, np.ndarray) else _torch().empty(
                self.n, dtype=b.dtype, device=b.device)
        _check_vec(x, self.n, "x")
        if se is not None:
            _check_vec(se, self.n, "se")
        res = Result()
        rc = lib().gsr_lsqr_solve(self._h, _ptr(b)[0], int(itmax), float(atol), float(btol),
                                  _ptr(x)[0], _ptr(se)[0] if se is not None else None,
                                  ctypes.byref(res), _stream(stream))
        check(rc, "gsr_lsqr_solve")
        return x, se, res.as_dict()
