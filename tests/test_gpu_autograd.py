"""Differentiable solve: the adjoint (normal-equation) solve against dense
linear algebra, gradients against a dense reference on the 1,000-star system
and against central finite differences (step 1e-6), including the full
medium-size system with the paper-style loss (gamma plus 1,000 parallaxes)."""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import gen
from tests._dense import columns, small

torch = pytest.importorskip("torch")
sparse = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _solver(sys):
    from paper_2212_11675_gb300.solver import Solver
    return Solver(sys, conlim=0.0)


def _sparse_A(sys):
    rows = np.repeat(np.arange(sys.m), 24)
    return sparse.csr_matrix((sys.values.ravel(), (rows, columns(sys).ravel())), shape=(sys.m, sys.n))


def _loss_weights(sys, nstars, seed=4242):
    """dL/dx for L = gamma + sum of the parallaxes of `nstars` random stars."""
    rng = np.random.default_rng(seed)
    stars = rng.choice(sys.n_stars, size=nstars, replace=False)
    g = np.zeros(sys.n)
    g[5 * stars] = 1.0
    g[5 * sys.n_stars + 3 * sys.n_dfa + sys.n_instr] = 1.0
    return g


def test_normal_solve_matches_dense():
    sys = small(60, 20, 12, seed=2)
    A = _sparse_A(sys).toarray()
    rng = np.random.default_rng(0)
    g = rng.standard_normal(sys.n)
    ref = np.linalg.solve(A.T @ A, g)
    with _solver(sys) as s:
        q, info = s.normal_solve(torch.tensor(g, device=DEV), max_iter=2000, tol=1e-14)
        q = q.cpu().numpy()
    assert np.linalg.norm(q - ref) <= 1e-9 * np.linalg.norm(ref), info


def _dense_gradients(sys, b, g):
    A = _sparse_A(sys)
    AtA = (A.T @ A).toarray()
    x = np.linalg.solve(AtA, A.T @ b)
    q = np.linalg.solve(AtA, g)
    s = A @ q
    r = b - A @ x
    G = sys.n - 1
    return x, s, r * q[G] - s * x[G]


def test_backward_matches_dense_reference_on_1000_stars():
    sys = gen.make("tiny")   # 1,000 stars, D = 200, I = 60
    xt = gen.x_true(sys, 7)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 8)
    g = _loss_weights(sys, 300)
    x_ref, gb_ref, ga_ref = _dense_gradients(sys, b, g)
    from paper_2212_11675_gb300.autograd import GsrSolve
    with _solver(sys) as s:
        bt = torch.tensor(b, device=DEV, requires_grad=True)
        at = torch.tensor(sys.values[:, 23].copy(), device=DEV, requires_grad=True)
        x = GsrSolve.apply(bt, at, s)
        loss = (x * torch.tensor(g, device=DEV)).sum()
        loss.backward()
        xs, gb, ga = x.detach().cpu().numpy(), bt.grad.cpu().numpy(), at.grad.cpu().numpy()
    assert np.linalg.norm(xs - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert np.linalg.norm(gb - gb_ref) <= 1e-8 * np.linalg.norm(gb_ref)
    assert np.linalg.norm(ga - ga_ref) <= 1e-8 * np.linalg.norm(ga_ref)


def _fd_check(sys, b, g, nb, na, seed, rtol):
    from paper_2212_11675_gb300.autograd import GsrSolve
    rng = np.random.default_rng(seed)
    a0 = sys.values[:, 23].copy()
    gt = torch.tensor(g, device=DEV)
    with _solver(sys) as s:
        bt = torch.tensor(b, device=DEV, requires_grad=True)
        at = torch.tensor(a0, device=DEV, requires_grad=True)
        loss = (GsrSolve.apply(bt, at, s) * gt).sum()
        loss.backward()
        gb, ga = bt.grad.cpu().numpy(), at.grad.cpu().numpy()

        def L(bv, av):
            with torch.no_grad():
                return float((GsrSolve.apply(torch.tensor(bv, device=DEV),
                                             torch.tensor(av, device=DEV), s) * gt).sum())

        h = 1e-6
        scale_b = np.abs(gb).max()
        for i in rng.choice(sys.m, size=nb, replace=False):
            bp, bm = b.copy(), b.copy()
            bp[i] += h
            bm[i] -= h
            fd = (L(bp, a0) - L(bm, a0)) / (2 * h)
            assert abs(fd - gb[i]) <= rtol * max(abs(gb[i]), 0.01 * scale_b), (i, fd, gb[i])
        scale_a = np.abs(ga).max()
        for i in rng.choice(sys.m, size=na, replace=False):
            ap, am = a0.copy(), a0.copy()
            ap[i] += h
            am[i] -= h
            fd = (L(b, ap) - L(b, am)) / (2 * h)
            assert abs(fd - ga[i]) <= rtol * max(abs(ga[i]), 0.01 * scale_a), (i, fd, ga[i])


def test_gradients_match_finite_differences_tiny():
    sys = gen.make("tiny")
    xt = gen.x_true(sys, 9)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 10)
    _fd_check(sys, b, _loss_weights(sys, 300), nb=8, na=8, seed=1, rtol=1e-4)


def test_gradients_match_finite_differences_medium():
    """The medium system (100,000 stars, ~7e6 rows) with the loss of the
    differentiated workload: gamma plus the parallaxes of 1,000 random stars."""
    sys = gen.make("medium")
    xt = gen.x_true(sys, 11)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 12)
    _fd_check(sys, b, _loss_weights(sys, 1000), nb=4, na=4, seed=2, rtol=1e-4)
