"""gsr_aprod1_norm_noalloc, the entry point for callers that cannot allocate
device memory at call time, checked through the C ABI against gsr_aprod1.

It computes y = A x + cy y and ||y|| with its scratch in a static device
array; with cy = 1 its y must equal gsr_aprod1's y += A x within the bound
the other product tests use (1e-12 of sum |terms| per element), and its norm
must be the norm of that vector.  Two calls in a row check that the shared
scratch (cleared counter, reused partial sums) carries nothing over.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import _lib, gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _bound(sys, x, y0):
    a = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff, sys.instr,
                       np.abs(sys.values))
    return 1e-12 * (oracle.aprod1(a, np.abs(x)) + np.abs(y0)) + 1e-300


def test_noalloc_matches_aprod1_on_two_calls_in_a_row():
    from paper_2212_11675_gb300.solver import Solver
    L = _lib.lib()
    sys = gen.make("tiny")
    rng = np.random.default_rng(21)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with Solver(sys) as s:
        for call in range(2):
            x = rng.standard_normal(sys.n)
            y0 = rng.standard_normal(sys.m)
            xd = torch.tensor(x, device="cuda")
            y_ref = torch.tensor(y0, device="cuda")
            _lib.check(L.gsr_aprod1(s.handle, _p(xd), _p(y_ref), stream), "gsr_aprod1")
            y = torch.tensor(y0, device="cuda")
            nrm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            _lib.check(L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), _p(y), ctypes.c_double(1.0),
                                                 _p(nrm), stream), "gsr_aprod1_norm_noalloc")
            torch.cuda.synchronize()
            g, r = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.all(np.abs(g - r) <= _bound(sys, x, y0)), call
            assert float(nrm) == pytest.approx(float(np.linalg.norm(r)), rel=1e-12), call


def test_noalloc_scaled_form_and_host_norm():
    """cy != 1 against gsr_aprod1 applied to cy*y; the norm into host memory."""
    from paper_2212_11675_gb300.solver import Solver
    L = _lib.lib()
    sys = gen.make("tiny")
    rng = np.random.default_rng(5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cy = -0.625
    with Solver(sys) as s:
        x = rng.standard_normal(sys.n)
        y0 = rng.standard_normal(sys.m)
        xd = torch.tensor(x, device="cuda")
        y_ref = torch.tensor(cy * y0, device="cuda")
        _lib.check(L.gsr_aprod1(s.handle, _p(xd), _p(y_ref), stream), "gsr_aprod1")
        y = torch.tensor(y0, device="cuda")
        host_norm = ctypes.c_double(-1.0)
        _lib.check(L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), _p(y), ctypes.c_double(cy),
                                             ctypes.byref(host_norm), stream),
                   "gsr_aprod1_norm_noalloc")
        torch.cuda.synchronize()
        g, r = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.abs(g - r) <= _bound(sys, x, cy * y0))
        assert host_norm.value == pytest.approx(float(np.linalg.norm(r)), rel=1e-12)
        # host vectors are refused (they would need staging memory)
        yh = np.zeros(sys.m)
        rc = L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), ctypes.c_void_p(yh.ctypes.data),
                                       ctypes.c_double(1.0), ctypes.byref(host_norm), stream)
        assert rc == _lib.GSR_ERR_ARG
