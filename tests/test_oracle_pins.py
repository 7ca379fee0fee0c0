"""Pins of the CPU oracle against facts fixed outside it.

Each test checks the oracle against something other than its own formula:
a hand-derived fixture, dense linear algebra, an identity, SciPy's independent
LSQR, LAPACK least squares or a textbook closed form.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import gen
from tests._dense import columns, dense, small

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_colmap():
    rows, cols = [], []
    with open(os.path.join(GOLDEN, "colmap_tiny.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("S "):
                t = line.split()
                S, D, I = int(t[1]), int(t[3]), int(t[5])
                continue
            left, right = line.split("|")
            rows.append([int(v) for v in left.split()])
            cols.append([int(v) for v in right.split()])
    rows = np.array(rows)
    stars = rows[:, 1]
    star_ptr = np.zeros(S + 1, dtype=np.uint32)
    for s in stars:
        star_ptr[s + 1:] += 1
    sys = gen.GaiaSystem(S, D, I, star_ptr, rows[:, 2].astype(np.uint32),
                         rows[:, 3:9].astype(np.uint16),
                         np.array([[100.0 * (r + 1) + k for k in range(24)] for r in range(len(rows))]))
    return sys, np.array(cols)


def test_golden_column_map():
    """Paper §3 layout: the oracle's products hit exactly the hand-derived columns."""
    sys, cols = _load_colmap()
    assert sys.n == 33
    A = np.zeros((sys.m, sys.n))
    for r in range(sys.m):
        for k in range(24):
            A[r, cols[r, k]] += sys.values[r, k]
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(sys.n)
        y = rng.standard_normal(sys.m)
        np.testing.assert_allclose(oracle.aprod1(sys, x), A @ x, rtol=1e-14, atol=1e-11)
        np.testing.assert_allclose(oracle.aprod2(sys, y), A.T @ y, rtol=1e-14, atol=1e-11)
    # unit vectors recover single columns exactly
    for j in (0, 9, 10, 14, 24, 25, 31, 32):
        e = np.zeros(sys.n)
        e[j] = 1.0
        np.testing.assert_array_equal(oracle.aprod1(sys, e), A[:, j])


@pytest.mark.parametrize("S,D,I,obs", [(7, 6, 9, 5), (40, 20, 10, None), (1, 4, 6, 3)])
def test_dense_bruteforce(S, D, I, obs):
    sys = small(S, D, I, obs)
    A = dense(sys)
    rng = np.random.default_rng(S)
    x = rng.standard_normal(sys.n)
    y = rng.standard_normal(sys.m)
    y0 = rng.standard_normal(sys.m)
    x0 = rng.standard_normal(sys.n)
    np.testing.assert_allclose(oracle.aprod1(sys, x, y0), y0 + A @ x, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(oracle.aprod2(sys, y, x0), x0 + A.T @ y, rtol=1e-13, atol=1e-12)


def test_adjoint_identity_tiny_config():
    sys = gen.make("tiny")
    rng = np.random.default_rng(1)
    x = rng.standard_normal(sys.n)
    y = rng.standard_normal(sys.m)
    ax = oracle.aprod1(sys, x)
    aty = oracle.aprod2(sys, y)
    lhs, rhs = ax @ y, x @ aty
    scale = np.linalg.norm(ax) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-13 * scale


def test_all_ones_gives_24():
    sys = gen.make("tiny")
    sys.values = np.ones_like(sys.values)
    y = oracle.aprod1(sys, np.ones(sys.n))
    np.testing.assert_array_equal(y, np.full(sys.m, 24.0))
    # column counts: A^T 1 counts the nonzeros of every column
    cnt = oracle.aprod2(sys, np.ones(sys.m))
    expect = np.bincount(columns(sys).ravel(), minlength=sys.n).astype(float)
    np.testing.assert_array_equal(cnt, expect)


def test_preconditioner_unit_columns_and_empty_column():
    # I = 40 with few rows leaves some instruments unobserved: their p must be 1
    sys = small(6, 8, 40, obs=3)
    A = dense(sys)
    p, scaled = oracle.precondition(sys)
    norms = np.linalg.norm(A, axis=0)
    used = norms > 0
    assert (~used).any()
    np.testing.assert_allclose(p[used], 1.0 / norms[used], rtol=1e-15)
    np.testing.assert_array_equal(p[~used], 1.0)
    As = dense(sys, scaled)
    np.testing.assert_allclose(np.linalg.norm(As, axis=0)[used], 1.0, rtol=1e-14)
    np.testing.assert_allclose(oracle.colnorms(sys), norms, rtol=1e-15)


def _rhs(sys, seed=3, sigma=1e-3):
    xt = gen.x_true(sys, seed)
    return xt, oracle.aprod1(sys, xt) + gen.noise(sys, seed + 1, sigma)


def test_lsqr_iterates_match_scipy():
    """P&S LSQR recurrences: iterate, var, anorm, acond, arnorm after k steps
    equal SciPy's independent implementation (damp=0)."""
    scipy_lsqr = pytest.importorskip("scipy.sparse.linalg").lsqr
    sys = small(30, 12, 8)
    A = dense(sys)
    _, b = _rhs(sys)
    for k in (1, 2, 5, 8):
        r = oracle.lsqr(sys, b, k, atol=0.0, btol=0.0, conlim=0.0)
        ref = scipy_lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k, calc_var=True)
        x_s, istop_s, itn_s, r1, r2, anorm_s, acond_s, arnorm_s, xnorm_s, var_s = ref
        assert r["itn"] == itn_s == k
        assert r["istop"] == 7
        np.testing.assert_allclose(r["z"], x_s, rtol=1e-11, atol=1e-12 * np.abs(x_s).max())
        np.testing.assert_allclose(r["var"], var_s, rtol=1e-11)
        assert r["rnorm"] == pytest.approx(r1, rel=1e-12)
        assert r["anorm"] == pytest.approx(anorm_s, rel=1e-13)
        assert r["acond"] == pytest.approx(acond_s, rel=1e-12)
        assert r["arnorm"] == pytest.approx(arnorm_s, rel=1e-10)


def test_lsqr_stopping_rules_match_scipy():
    """S1 (btol/atol on rnorm) fires at the same iteration as SciPy; S2 fires
    within a few iterations (arnorm is not monotone, so rounding can move the
    crossing of a threshold by one or two steps)."""
    scipy_lsqr = pytest.importorskip("scipy.sparse.linalg").lsqr
    sys = small(30, 12, 8)
    A = dense(sys)
    _, b = _rhs(sys)
    r = oracle.lsqr(sys, b, 1000, atol=1e-4, btol=0.0, conlim=0.0)
    ref = scipy_lsqr(A, b, atol=1e-4, btol=0.0, conlim=0.0, iter_lim=1000)
    assert r["istop"] == ref[1] == 1
    assert r["itn"] == ref[2]
    r = oracle.lsqr(sys, b, 1000, atol=1e-6, btol=0.0, conlim=0.0)
    ref = scipy_lsqr(A, b, atol=1e-6, btol=0.0, conlim=0.0, iter_lim=1000)
    assert r["istop"] == ref[1] == 2
    assert abs(r["itn"] - ref[2]) <= 3
    # S3: a tiny condition limit stops on acond
    r = oracle.lsqr(sys, b, 1000, atol=0.0, btol=0.0, conlim=2.0)
    ref = scipy_lsqr(A, b, atol=0.0, btol=0.0, conlim=2.0, iter_lim=1000)
    assert r["istop"] == ref[1] == 3
    assert r["itn"] == ref[2]


def test_lsqr_machine_precision_rules_match_scipy():
    """Rules 4 and 5 (S1 and S2 with the tolerance at machine precision) fire
    as in SciPy: with atol = btol = 0 and no condition limit, a consistent
    system stops on rule 4 and an inconsistent one on rule 5, within a few
    iterations of SciPy (the last iterations are rounding-dominated).  Rule 6
    (the condition estimate beyond 1/eps) is not pinned: on these shapes
    rule 5 fires first in both implementations."""
    scipy_lsqr = pytest.importorskip("scipy.sparse.linalg").lsqr
    sys = small(30, 12, 8, seed=3)
    A = dense(sys)
    rng = np.random.default_rng(1)
    b = A @ rng.standard_normal(sys.n)
    r = oracle.lsqr(sys, b, 2000, atol=0.0, btol=0.0, conlim=0.0)
    ref = scipy_lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=2000)
    assert r["istop"] == ref[1] == 4
    assert abs(r["itn"] - ref[2]) <= 5
    b = b + 1e-3 * rng.standard_normal(sys.m)
    r = oracle.lsqr(sys, b, 2000, atol=0.0, btol=0.0, conlim=0.0)
    ref = scipy_lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=2000)
    assert r["istop"] == ref[1] == 5
    assert abs(r["itn"] - ref[2]) <= 5


def test_run_to_itmax_changes_no_arithmetic():
    """run_to_itmax only keeps the loop going: up to the iteration where a
    rule fires, the iterates are bit-identical to a run that stops there, and
    past it they equal a run with every rule switched off."""
    sys = small(30, 12, 8)
    _, b = _rhs(sys)
    stop = oracle.pc_lsqr(sys, b, 1000, atol=1e-6, btol=0.0, conlim=0.0)
    assert stop["istop"] == 2 and stop["itn"] < 200
    k = stop["itn"]
    same = oracle.pc_lsqr(sys, b, k, atol=1e-6, btol=0.0, conlim=0.0, run_to_itmax=True)
    np.testing.assert_array_equal(same["x"], stop["x"])
    assert same["itn"] == k and same["istop"] == 2
    longer = oracle.pc_lsqr(sys, b, k + 30, atol=1e-6, btol=0.0, conlim=0.0, run_to_itmax=True)
    free = oracle.pc_lsqr(sys, b, k + 30, atol=0.0, btol=0.0, conlim=0.0, run_to_itmax=True)
    assert longer["itn"] == free["itn"] == k + 30
    np.testing.assert_array_equal(longer["x"], free["x"])
    np.testing.assert_array_equal(longer["se"], free["se"])


def test_pc_lsqr_matches_lapack_lstsq():
    sys = small(30, 12, 8)
    A = dense(sys)
    _, b = _rhs(sys)
    r = oracle.pc_lsqr(sys, b, 2000, atol=1e-15, btol=1e-15, conlim=1e12)
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(r["x"] - x_ls) <= 1e-10 * np.linalg.norm(x_ls)
    # the rnorm estimate is the true residual norm of the returned solution
    res = np.linalg.norm(b - A @ r["x"])
    assert r["rnorm"] == pytest.approx(res, rel=1e-10)


def test_pc_lsqr_recovers_x_true_noise_free():
    sys = small(50, 16, 10)
    xt = gen.x_true(sys, 11)
    b = dense(sys) @ xt
    r = oracle.pc_lsqr(sys, b, 5000, atol=1e-15, btol=1e-15, conlim=1e12)
    assert r["istop"] in (1, 4)
    assert np.linalg.norm(r["x"] - xt) <= 1e-10 * np.linalg.norm(xt)


def test_rnorm_trace_invariants():
    """phibar is non-increasing and equals the explicit residual norm at every k;
    arnorm equals the explicit ||A_pc^T r||."""
    sys = small(40, 20, 10)
    A = dense(sys)
    _, b = _rhs(sys)
    full = oracle.pc_lsqr(sys, b, 60, atol=0.0, btol=0.0, conlim=0.0, trace=True)
    tr = full["trace_rnorm"]
    assert np.all(np.diff(tr) <= 1e-12 * tr[0])
    for k in (1, 3, 10, 25):
        r = oracle.pc_lsqr(sys, b, k, atol=0.0, btol=0.0, conlim=0.0)
        resid = b - A @ r["x"]
        assert r["rnorm"] == pytest.approx(np.linalg.norm(resid), rel=1e-10)
        assert r["rnorm"] == pytest.approx(tr[k - 1], rel=1e-14)
        arn = np.linalg.norm(r["p"] * (A.T @ resid))
        assert r["arnorm"] == pytest.approx(arn, rel=1e-7)


def test_standard_errors_reach_textbook_limit():
    """After n steps on a tiny full-rank system, var = diag((A_pc^T A_pc)^-1) and
    se = sigma_hat * sqrt(diag((A^T A)^-1)), sigma_hat^2 = ||r||^2/(m-n)."""
    sys = small(2, 5, 7, obs=40)
    A = dense(sys)
    m, n = A.shape
    _, b = _rhs(sys, sigma=1e-1)
    r = oracle.pc_lsqr(sys, b, n, atol=0.0, btol=0.0, conlim=0.0)
    x_ls, res, *_ = np.linalg.lstsq(A, b, rcond=None)
    sigma = np.sqrt(res[0] / (m - n))
    se_ref = sigma * np.sqrt(np.diag(np.linalg.inv(A.T @ A)))
    np.testing.assert_allclose(r["x"], x_ls, rtol=1e-9, atol=1e-9 * np.abs(x_ls).max())
    # finite-precision Lanczos loses some orthogonality: 1e-4 is far below the
    # errors a wrong factor (m vs m-n, a missing p or sqrt) would cause
    np.testing.assert_allclose(r["se"], se_ref, rtol=1e-4)


def test_zero_rhs_gives_istop_zero():
    sys = small(5, 6, 7)
    r = oracle.pc_lsqr(sys, np.zeros(sys.m), 10)
    assert r["istop"] == 0 and r["itn"] == 0
    assert not r["x"].any()


def test_single_precision_products_dense_restatement():
    """The binary32-product operator against a dense NumPy restatement:
    float32 elementwise products, summed in float64."""
    sys = small(20, 10, 9)
    cols = columns(sys)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(sys.n)
    y = rng.standard_normal(sys.m)
    a32 = sys.values.astype(np.float32)
    prod1 = (a32 * x.astype(np.float32)[cols]).astype(np.float64)      # float32 products
    np.testing.assert_allclose(oracle.aprod1_f32(sys, x), prod1.sum(axis=1), rtol=1e-14, atol=1e-13)
    prod2 = (a32 * y.astype(np.float32)[:, None]).astype(np.float64)
    ref2 = np.zeros(sys.n)
    np.add.at(ref2, cols.ravel(), prod2.ravel())
    np.testing.assert_allclose(oracle.aprod2_f32(sys, y), ref2, rtol=1e-13, atol=1e-12)


def test_single_precision_products_exact_on_small_integers():
    """Small-integer values and vectors have exact binary32 products: the
    binary32-product operator then equals the FP64 one exactly."""
    sys = small(15, 8, 7)
    rng = np.random.default_rng(6)
    sys.values = rng.integers(-7, 8, size=sys.values.shape).astype(np.float64)
    x = rng.integers(-9, 10, size=sys.n).astype(np.float64)
    y = rng.integers(-9, 10, size=sys.m).astype(np.float64)
    np.testing.assert_array_equal(oracle.aprod1_f32(sys, x), oracle.aprod1(sys, x))
    np.testing.assert_array_equal(oracle.aprod2_f32(sys, y), oracle.aprod2(sys, y))
    # and it differs from FP64 by single-precision rounding on general inputs
    sys2 = small(15, 8, 7)
    xg = rng.standard_normal(sys2.n)
    d = np.abs(oracle.aprod1_f32(sys2, xg) - oracle.aprod1(sys2, xg))
    assert 0 < d.max() < 1e-5 * np.abs(oracle.aprod1(sys2, xg)).max()
