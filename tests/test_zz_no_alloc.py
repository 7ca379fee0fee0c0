"""gsr_aprod1_norm_noalloc, the entry point for callers that cannot allocate
device memory at call time (another component owns the device-memory budget
through its own pool, or a cudaMalloc would synchronise the device where the
caller cannot afford it), checked through the C ABI.

It computes y = A x + cy y and ||y|| with its scratch in a static device
array.  Its y must equal the oracle's A x + cy y0 within the bound the other
product tests use (1e-12 of sum |terms| per element), and its norm must be
the norm of that vector.  Two calls in a row check that the shared scratch
(coefficient slot, cleared counter, reused partial sums) carries nothing
over, and the free device memory must not change across calls.  This file
is collected last, so a run that stops at the first failure has run every
other test first.
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


def _bound(sys, x, cy, y0):
    a = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff, sys.instr,
                       np.abs(sys.values))
    return 1e-12 * (oracle.aprod1(a, np.abs(x)) + np.abs(cy * y0)) + 1e-300


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("cy", [1.0, -0.625])
def test_noalloc_matches_oracle_on_two_calls_in_a_row(cy):
    from paper_2212_11675_gb300.solver import Solver
    L = _lib.lib()
    sys = gen.make("tiny")
    rng = np.random.default_rng(21)
    with Solver(sys) as s:
        for call in range(2):
            x = rng.standard_normal(sys.n)
            y0 = rng.standard_normal(sys.m)
            ref = oracle.aprod1(sys, x, cy * y0)
            xd = torch.tensor(x, device="cuda")
            y = torch.tensor(y0, device="cuda")
            nrm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            _lib.check(L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), _p(y), ctypes.c_double(cy),
                                                 _p(nrm), _stream()), "gsr_aprod1_norm_noalloc")
            torch.cuda.synchronize()
            g = y.cpu().numpy()
            assert np.all(np.abs(g - ref) <= _bound(sys, x, cy, y0)), call
            assert float(nrm) == pytest.approx(float(np.linalg.norm(ref)), rel=1e-11), call


def test_noalloc_host_norm_and_refusals():
    """The norm into host memory; host vectors are refused (they would need
    staging memory)."""
    from paper_2212_11675_gb300.solver import Solver
    L = _lib.lib()
    sys = gen.make("tiny")
    rng = np.random.default_rng(5)
    cy = -0.625
    with Solver(sys) as s:
        x = rng.standard_normal(sys.n)
        y0 = rng.standard_normal(sys.m)
        ref = oracle.aprod1(sys, x, cy * y0)
        xd = torch.tensor(x, device="cuda")
        y = torch.tensor(y0, device="cuda")
        host_norm = ctypes.c_double(-1.0)
        _lib.check(L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), _p(y), ctypes.c_double(cy),
                                             ctypes.byref(host_norm), _stream()),
                   "gsr_aprod1_norm_noalloc")
        torch.cuda.synchronize()
        assert np.all(np.abs(y.cpu().numpy() - ref) <= _bound(sys, x, cy, y0))
        assert host_norm.value == pytest.approx(float(np.linalg.norm(ref)), rel=1e-11)
        yh = np.zeros(sys.m)
        rc = L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), ctypes.c_void_p(yh.ctypes.data),
                                       ctypes.c_double(1.0), ctypes.byref(host_norm), _stream())
        assert rc == _lib.GSR_ERR_ARG


def test_noalloc_leaves_free_device_memory_unchanged():
    """The defining property: calls allocate nothing on the device.  Every
    tensor is created before the first measurement."""
    from paper_2212_11675_gb300.solver import Solver
    L = _lib.lib()
    sys = gen.make("tiny")
    rng = np.random.default_rng(9)
    with Solver(sys) as s:
        x = rng.standard_normal(sys.n)
        xd = torch.tensor(x, device="cuda")
        y = torch.zeros(sys.m, dtype=torch.float64, device="cuda")
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(4):
            _lib.check(L.gsr_aprod1_norm_noalloc(s.handle, _p(xd), _p(y), ctypes.c_double(0.0),
                                                 _p(nrm), _stream()), "gsr_aprod1_norm_noalloc")
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        ref = oracle.aprod1(sys, x)
        assert float(nrm) == pytest.approx(float(np.linalg.norm(ref)), rel=1e-11)
