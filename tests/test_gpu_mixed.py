"""Mixed-precision form: the binary32-product operator against the oracle's
definition of it, and the refined solution against the FP64 oracle.

Operator bound: both sides form the same binary32 products (IEEE round to
nearest); only their accumulation differs (double-float on the GPU, double in
the oracle), so element j agrees within 1e-12 of sum |products|.
Solution bar: the FP64 least-squares solution to 1e-9 relative (the oracle's
PC-LSQR run to atol = btol = 1e-14), and the FP64 residual norms.
"""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import _lib, gen
from tests._dense import small
from tests._systems import ragged

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _solver(sys, **kw):
    from paper_2212_11675_gb300.solver import Solver
    return Solver(sys, precision=_lib.GSR_PREC_MIXED, **kw)


def _abs(sys):
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                          sys.instr, np.abs(sys.values))


@pytest.mark.parametrize("which", ["tiny", "ragged", "wide_instr"])
def test_f32_operator_parity(which):
    sys = {"tiny": lambda: gen.make("tiny"), "ragged": lambda: ragged(seed=21),
           "wide_instr": lambda: small(200, 40, 7000, seed=3)}[which]()
    rng = np.random.default_rng(1)
    x = rng.standard_normal(sys.n)
    y = rng.standard_normal(sys.m)
    y0 = rng.standard_normal(sys.m)
    x0 = rng.standard_normal(sys.n)
    ref1 = oracle.aprod1_f32(sys, x, y0)
    ref2 = oracle.aprod2_f32(sys, y, x0)
    b1 = 1e-12 * (oracle.aprod1(_abs(sys), np.abs(x)) + np.abs(y0)) + 1e-300
    b2 = 1e-12 * (oracle.aprod2(_abs(sys), np.abs(y)) + np.abs(x0)) + 1e-300
    with _solver(sys) as s:
        yd = torch.tensor(y0, device=DEV)
        s.aprod1_f32(torch.tensor(x, device=DEV), yd)
        xd = torch.tensor(x0, device=DEV)
        s.aprod2_f32(torch.tensor(y, device=DEV), xd)
        g1, g2 = yd.cpu().numpy(), xd.cpu().numpy()
    assert np.all(np.abs(g1 - ref1) <= b1), np.max(np.abs(g1 - ref1) / b1)
    assert np.all(np.abs(g2 - ref2) <= b2), np.max(np.abs(g2 - ref2) / b2)


def _fp64_solution(sys, b):
    return oracle.pc_lsqr(sys, b, 5000, 1e-14, 1e-14, conlim=1e12)


# The least-squares solution is unique only for full column rank (every star
# observed at least 5 times); refinement with a binary32 inner operator does
# not keep a rank-deficient iterate on the minimum-norm solution.
@pytest.mark.parametrize("which", ["tiny", "uneven"])
def test_mixed_solve_reaches_fp64_solution(which):
    sys = gen.make("tiny") if which == "tiny" else small(257, 37, 11, seed=31)
    xt = gen.x_true(sys, 3)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 4)
    ref = _fp64_solution(sys, b)
    with _solver(sys) as s:
        x, res = s.mixed_solve(torch.tensor(b, device=DEV), max_outer=20, max_inner=200,
                               inner_tol=1e-5, atol=1e-13)
        x = x.cpu().numpy()
    assert res["converged"] == 1, res
    assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"]), res
    assert res["rnorm"] == pytest.approx(np.linalg.norm(b - oracle.aprod1(sys, x)), rel=1e-9)
    assert res["rnorm"] == pytest.approx(ref["rnorm"], rel=1e-9)


def test_mixed_solve_host_buffers_and_errors():
    sys = small(300, 29, 13, seed=33)
    xt = gen.x_true(sys, 5)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 6)
    ref = _fp64_solution(sys, b)
    with _solver(sys) as s:
        x, res = s.mixed_solve(b, max_outer=20, max_inner=200, inner_tol=1e-5, atol=1e-13)
        assert isinstance(x, np.ndarray) and res["converged"] == 1
        assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])
        bad = b.copy()
        bad[3] = np.inf
        with pytest.raises(_lib.GsrError) as e:
            s.mixed_solve(bad)
        assert e.value.code == _lib.GSR_ERR_NONFINITE
    from paper_2212_11675_gb300.solver import Solver
    with Solver(sys) as s64:   # an FP64-only handle has no binary32 copy
        with pytest.raises(_lib.GsrError) as e:
            s64.mixed_solve(b)
        assert e.value.code == _lib.GSR_ERR_UNSUPPORTED


@pytest.mark.parametrize("mode,fused", [(_lib.GSR_INSTR_SORTED, False), (_lib.GSR_INSTR_SMEM, None),
                                        (_lib.GSR_INSTR_REPLICAS, None)])
def test_mixed_solve_other_schedules(mode, fused):
    # the inner solve's aprod 2 as separate launches, and on the shared-memory
    # and replica instrumental paths (the inner CG graph is captured again
    # when the schedule changes)
    sys = small(257, 37, 11, seed=31)
    xt = gen.x_true(sys, 3)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 4)
    ref = _fp64_solution(sys, b)
    with _solver(sys, instr_mode=mode) as s:
        if fused is not None:
            s.set_aprod2_fused(fused)
        x, res = s.mixed_solve(torch.tensor(b, device=DEV), max_outer=20, max_inner=200,
                               inner_tol=1e-5, atol=1e-13)
        x = x.cpu().numpy()
    assert res["converged"] == 1, res
    assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"]), res
