"""Batched k right-hand-side form: its skinny products against the oracle's
binary32-product operator column by column, and its solutions against the
FP64 least-squares solutions of every right-hand side."""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import _lib, gen
from tests._dense import small

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _solver(sys):
    from paper_2212_11675_gb300.solver import Solver
    return Solver(sys, precision=_lib.GSR_PREC_MIXED, conlim=0.0)


def _abs(sys):
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                          sys.instr, np.abs(sys.values))


@pytest.mark.parametrize("k,kt,lanes", [(5, 8, 16), (11, 4, 8), (3, 1, 32), (8, 2, 16)])
def test_batched_products_match_oracle(k, kt, lanes):
    sys = gen.make("tiny")
    rng = np.random.default_rng(k)
    X = rng.standard_normal((k, sys.n))
    Y = rng.standard_normal((k, sys.m))
    with _solver(sys) as s:
        s.set_batch_tiling(kt, lanes)
        Q, T = s.batched_products(torch.tensor(X, device=DEV), torch.tensor(Y, device=DEV))
        Q, T = Q.cpu().numpy(), T.cpu().numpy()
    a = _abs(sys)
    for c in range(k):
        r1 = oracle.aprod1_f32(sys, X[c])
        r2 = oracle.aprod2_f32(sys, Y[c])
        b1 = 1e-12 * oracle.aprod1(a, np.abs(X[c])) + 1e-300
        b2 = 1e-12 * oracle.aprod2(a, np.abs(Y[c])) + 1e-300
        # Q is stored in binary32 (it feeds the next binary32 product): half an
        # ulp of binary32 on top of the accumulation bound
        half_ulp = 0.5 * np.spacing(np.abs(r1).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(Q[c] - r1) <= b1 + half_ulp), c
        assert np.all(np.abs(T[c] - r2) <= b2), (c, np.max(np.abs(T[c] - r2) / b2))


@pytest.mark.parametrize("k", [3, 10])
def test_batched_solve_matches_fp64_solutions(k):
    sys = small(257, 37, 11, seed=31)   # full column rank
    xt = gen.x_true(sys, 3)
    ax = oracle.aprod1(sys, xt)
    B = np.stack([ax + gen.noise(sys, 100 + j) for j in range(k)])
    with _solver(sys) as s:
        X, res = s.batched_solve(torch.tensor(B, device=DEV), max_outer=20, max_inner=300,
                                 inner_tol=1e-5, atol=1e-13)
        X = X.cpu().numpy()
    for j in range(k):
        ref = oracle.pc_lsqr(sys, B[j], 5000, 1e-14, 1e-14, conlim=1e12)
        assert res[j]["converged"] == 1, (j, res[j])
        assert np.linalg.norm(X[j] - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"]), j
        assert res[j]["rnorm"] == pytest.approx(ref["rnorm"], rel=1e-9)


def test_batched_solve_host_buffers_tiny():
    sys = gen.make("tiny")
    xt = gen.x_true(sys, 5)
    ax = oracle.aprod1(sys, xt)
    B = np.stack([ax + gen.noise(sys, 200 + j) for j in range(4)])
    with _solver(sys) as s:
        s.set_batch_tiling(4, 16)
        X, res = s.batched_solve(B, max_outer=20, max_inner=300, inner_tol=1e-5, atol=1e-13)
    for j in range(4):
        ref = oracle.pc_lsqr(sys, B[j], 5000, 1e-14, 1e-14, conlim=1e12)
        assert np.linalg.norm(X[j] - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])
