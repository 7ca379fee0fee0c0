"""aprod 1 with the instrumental and global products on the binary32 pipes
(GSR_PRODUCTS_SPLIT, the default where I <= 3072) against exact rational
arithmetic: the split products are accumulated to within about 2^-60 of the
sum of their magnitudes, so a row made only of them stays accurate under
heavy cancellation, where a chain of FP64 FMAs loses up to 2^-53 of that sum
per product.  Operands outside the split range take the native FP64
products; the result then meets the FP64 bound."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2212_11675_gb300 import _lib, gen
from tests._dense import columns, small

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
U = 2.0 ** -53


def _exact(sys, x, y0):
    """y0 + A x row by row in rational arithmetic, and sum |terms|."""
    cols = columns(sys)
    ex, mag = [], []
    for i in range(sys.m):
        t = Fraction(float(y0[i]))
        s = abs(float(y0[i]))
        for k in range(24):
            p = Fraction(float(sys.values[i, k])) * Fraction(float(x[cols[i, k]]))
            t += p
            s += abs(float(p))
        ex.append(t)
        mag.append(s)
    return ex, np.array(mag)


def _aprod1(sys, x, y0, products):
    from paper_2212_11675_gb300.solver import Solver
    with Solver(sys, products=products) as s:
        yd = torch.tensor(y0, device=DEV)
        s.aprod1(torch.tensor(x, device=DEV), yd)
        return yd.cpu().numpy()


def _err(g, ex):
    return np.array([abs(float(Fraction(float(v)) - e)) for v, e in zip(g, ex)])


def _cancelling_system(seed):
    """Rows whose astrometric and attitude values are zero and whose seven
    instrumental and global products (about 2^49 in magnitude) cancel: the
    global value is minus the instrumental sum over the global x, rounded,
    so the exact row sum is that rounding residual, near 2^-3."""
    sys = small(40, 12, 9, obs=8, seed=seed)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(sys.n)
    ins0 = 5 * sys.n_stars + 3 * sys.n_dfa
    x[ins0:] = rng.uniform(1.0, 2.0, size=sys.n - ins0) * 2.0 ** 24
    vals = sys.values.copy()
    vals[:, :17] = 0.0
    sign = np.where(np.arange(6) % 2 == 0, 1.0, -1.0)
    vals[:, 17:23] = rng.uniform(1.0, 2.0, size=(sys.m, 6)) * 2.0 ** 24 * sign[None, :]
    xg = Fraction(float(x[-1]))
    for i in range(sys.m):
        part = sum(Fraction(float(vals[i, 17 + j])) * Fraction(float(x[ins0 + int(sys.instr[i, j])]))
                   for j in range(6))
        vals[i, 23] = -float(part / xg)
    cancel = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                            sys.instr, vals)
    return cancel, x


def test_split_products_exact_under_cancellation():
    sys, x = _cancelling_system(3)
    y0 = np.zeros(sys.m)
    ex, mag = _exact(sys, x, y0)
    exf = np.array([float(e) for e in ex])
    assert np.median(mag / np.maximum(np.abs(exf), 1e-300)) > 1e6  # real cancellation
    g = _aprod1(sys, x, y0, _lib.GSR_PRODUCTS_SPLIT)
    # the final binary64 roundings plus 2^-60 of sum |terms|
    assert np.all(_err(g, ex) <= 2 * U * np.abs(exf) + 2.0 ** -60 * mag)
    gn = _aprod1(sys, x, y0, _lib.GSR_PRODUCTS_NATIVE)
    # the FP64 chain meets only its own bound, far looser here
    assert np.all(_err(gn, ex) <= 30 * U * mag)
    assert np.max(_err(gn, ex) / np.maximum(np.abs(exf), 1e-300)) > 1e-12


@pytest.mark.parametrize("products", [_lib.GSR_PRODUCTS_SPLIT, _lib.GSR_PRODUCTS_NATIVE])
def test_split_and_native_meet_the_fp64_bound(products):
    sys = small(60, 20, 13, obs=12, seed=4)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    ex, mag = _exact(sys, x, y0)
    g = _aprod1(sys, x, y0, products)
    # gamma_27 over the 24 products, the chain merge and the y0 term
    assert np.all(_err(g, ex) <= 27 * U * mag)


def test_split_out_of_range_operands_fall_back():
    sys = small(60, 20, 13, obs=12, seed=6)
    rng = np.random.default_rng(7)
    vals = sys.values.copy()
    vals[0, 17] = 1e-12       # below 2^-30
    vals[1, 20] = 3e12        # above 2^30
    vals[2, 23] = 0.0         # zero value
    vals[3, 18] = 2.0 ** -30  # smallest in range
    vals[4, 19] = -(2.0 ** 31) * (1 - 2.0 ** -53)  # largest in range
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    ins0 = 5 * sys.n_stars + 3 * sys.n_dfa
    x[ins0 + 2] = 0.0  # a zero instrumental x is split exactly
    for case in range(3):
        xc = x.copy()
        if case == 1:
            xc[ins0 + 5] = 1e-14  # instrumental x out of range: native for every row
        if case == 2:
            xc[-1] = 1e15         # global x out of range
        ex, mag = _exact(sys, xc, y0)
        g = _aprod1(sys, xc, y0, _lib.GSR_PRODUCTS_SPLIT)
        assert np.all(_err(g, ex) <= 27 * U * mag), case


def test_split_matches_native_on_a_generated_system():
    sys = gen.make("tiny")
    rng = np.random.default_rng(9)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    gs = _aprod1(sys, x, y0, _lib.GSR_PRODUCTS_SPLIT)
    gn = _aprod1(sys, x, y0, _lib.GSR_PRODUCTS_NATIVE)
    a = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                       sys.instr, np.abs(sys.values))
    cols = columns(a)
    mag = np.abs(y0) + np.sum(a.values * np.abs(x)[cols], axis=1)
    assert np.all(np.abs(gs - gn) <= 54 * U * mag)
    assert not np.array_equal(gs, gn)  # the two forms really differ in rounding
