"""The split product forms (GSR_PRODUCTS_SPLIT and the GSR_PRODUCTS_MASK
choices; aprod 1's is the default where I <= 3072) against exact rational
arithmetic: the split products are
accumulated to within about 2^-60 of the sum of their magnitudes, so a row
(or a star's column sum) made only of them stays accurate under heavy
cancellation, where a chain of FP64 FMAs loses up to 2^-53 of that sum per
product.  Operands outside the split range take the native FP64 products;
the result then meets the FP64 bound."""
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
    uses5 = (sys.instr == 5).any(axis=1)
    assert uses5.any() and not uses5.all()
    g0 = None
    for case in range(3):
        xc = x.copy()
        if case == 1:
            xc[ins0 + 5] = 1e-14  # instrumental x out of range: native for the rows using it
        if case == 2:
            xc[-1] = 1e15         # global x out of range: native for every row
        ex, mag = _exact(sys, xc, y0)
        g = _aprod1(sys, xc, y0, _lib.GSR_PRODUCTS_SPLIT)
        assert np.all(_err(g, ex) <= 27 * U * mag), case
        if case == 0:
            g0 = g
        if case == 1:
            # the other rows keep their split products: identical to case 0
            np.testing.assert_array_equal(g[~uses5], g0[~uses5])


ASTRO = _lib.GSR_PRODUCTS_MASK | _lib.GSR_SPLIT_APROD1 | _lib.GSR_SPLIT_APROD1_ASTRO


def test_split_astrometric_products_exact_under_cancellation():
    # rows whose attitude values are zero and whose 12 astrometric,
    # instrumental and global products (about 2^48 each) cancel to a rounding
    # residual: with the astrometric products also split (staged aprod 1),
    # the row is within the final roundings plus 2^-60 of sum |terms|
    sys = small(40, 12, 9, obs=8, seed=41)
    rng = np.random.default_rng(41)
    x = rng.standard_normal(sys.n)
    ins0 = 5 * sys.n_stars + 3 * sys.n_dfa
    x[:5 * sys.n_stars] = rng.uniform(1.0, 2.0, size=5 * sys.n_stars) * 2.0 ** 24
    x[ins0:] = rng.uniform(1.0, 2.0, size=sys.n - ins0) * 2.0 ** 24
    vals = sys.values.copy()
    vals[:, 5:17] = 0.0
    sign = np.where(np.arange(11) % 2 == 0, 1.0, -1.0)
    big = rng.uniform(1.0, 2.0, size=(sys.m, 11)) * 2.0 ** 24 * sign[None, :]
    vals[:, 0:5] = big[:, :5]
    vals[:, 17:23] = big[:, 5:]
    cols = columns(sys)
    xg = Fraction(float(x[-1]))
    for i in range(sys.m):
        part = sum(Fraction(float(vals[i, k])) * Fraction(float(x[cols[i, k]]))
                   for k in list(range(5)) + list(range(17, 23)))
        vals[i, 23] = -float(part / xg)
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    from paper_2212_11675_gb300.solver import Solver
    with Solver(sys, products=ASTRO) as s:
        assert s.aprod1_staging() and s.product_forms()[0] == 2
    y0 = np.zeros(sys.m)
    ex, mag = _exact(sys, x, y0)
    exf = np.array([float(e) for e in ex])
    assert np.median(mag / np.maximum(np.abs(exf), 1e-300)) > 1e6
    g = _aprod1(sys, x, y0, ASTRO)
    assert np.all(_err(g, ex) <= 2 * U * np.abs(exf) + 2.0 ** -60 * mag)
    # the default split form keeps the five astrometric FMAs native
    gd = _aprod1(sys, x, y0, _lib.GSR_PRODUCTS_SPLIT)
    assert np.all(_err(gd, ex) <= 30 * U * mag)
    assert np.max(_err(gd, ex) / np.maximum(np.abs(exf), 1e-300)) > 1e-12


def test_split_astrometric_out_of_range_fall_back():
    sys = small(60, 20, 13, obs=12, seed=42)
    rng = np.random.default_rng(43)
    vals = sys.values.copy()
    vals[0, 2] = 1e-12    # astrometric value below 2^-30
    vals[1, 4] = 3e12     # above 2^30
    vals[2, 0] = 0.0      # zero value
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    for case in range(3):
        xc = x.copy()
        if case == 1:
            xc[5 * 3 + 1] = 1e-14  # star 3's parallax out of range: its rows go native
        if case == 2:
            xc[5 * 7] = 0.0        # a zero x splits exactly
        ex, mag = _exact(sys, xc, y0)
        g = _aprod1(sys, xc, y0, ASTRO)
        assert np.all(_err(g, ex) <= 27 * U * mag), case


def test_split_astrometric_products_and_solve():
    from tests.test_gpu_parity import check_aprods, compare_solve
    from tests._systems import ragged
    for sys in (gen.make("tiny"), ragged()):
        check_aprods(sys, 8, products=ASTRO)
    compare_solve(gen.make("tiny"), 200, 1e-12, 1e-12, products=ASTRO)


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


def _exact_t(sys, y, x0):
    """x0 + A^T y column by column in rational arithmetic, and sum |terms|."""
    cols = columns(sys)
    ex = [Fraction(float(v)) for v in x0]
    mag = np.abs(x0).astype(float)
    for i in range(sys.m):
        yi = Fraction(float(y[i]))
        for k in range(24):
            p = Fraction(float(sys.values[i, k])) * yi
            ex[cols[i, k]] += p
            mag[cols[i, k]] += abs(float(p))
    return ex, mag


def _aprod2(sys, y, x0, products):
    from paper_2212_11675_gb300.solver import Solver
    with Solver(sys, products=products, instr_mode=_lib.GSR_INSTR_SORTED) as s:
        xd = torch.tensor(x0, device=DEV)
        s.aprod2(torch.tensor(y, device=DEV), xd)
        return xd.cpu().numpy()


def test_split_star_sums_exact_under_cancellation():
    # aprod 2's astrometric sums: in every star the first astrometric value
    # of the last row cancels the star's other products of that column
    sys = small(40, 12, 9, obs=9, seed=11)
    rng = np.random.default_rng(11)
    vals = sys.values.copy()
    y = rng.uniform(1.0, 2.0, size=sys.m) * 2.0 ** 20 * np.where(np.arange(sys.m) % 2 == 0, 1, -1)
    vals[:, 0] = rng.uniform(1.0, 2.0, size=sys.m) * 2.0 ** 20
    sp = sys.star_ptr.astype(np.int64)
    for s in range(sys.n_stars):
        r0, r1 = sp[s], sp[s + 1]
        part = sum(Fraction(float(vals[r, 0])) * Fraction(float(y[r])) for r in range(r0, r1 - 1))
        vals[r1 - 1, 0] = -float(part / Fraction(float(y[r1 - 1])))
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x0 = np.zeros(sys.n)
    ex, mag = _exact_t(sys, y, x0)
    exf = np.array([float(e) for e in ex])
    c0 = 5 * np.arange(sys.n_stars)
    assert np.median(mag[c0] / np.maximum(np.abs(exf[c0]), 1e-300)) > 1e6
    g = _aprod2(sys, y, x0, _lib.GSR_PRODUCTS_SPLIT)
    err = _err(g, ex)
    astro = np.arange(5 * sys.n_stars)
    assert np.all(err[astro] <= 3 * U * np.abs(exf[astro]) + 2.0 ** -60 * mag[astro])
    assert np.all(err <= 30 * U * mag)
    gn = _aprod2(sys, y, x0, _lib.GSR_PRODUCTS_NATIVE)
    errn = _err(gn, ex)
    assert np.all(errn <= 30 * U * mag)
    assert np.max(errn[c0] / np.maximum(np.abs(exf[c0]), 1e-300)) > 1e-12


def test_split_star_sums_out_of_range_fall_back():
    sys = small(60, 20, 13, obs=12, seed=12)
    rng = np.random.default_rng(13)
    vals = sys.values.copy()
    vals[5, 2] = 1e-13   # astrometric value below the split range
    vals[40, 23] = 5e11  # global value above it
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x0 = rng.standard_normal(sys.n)
    for case in range(3):
        y = rng.standard_normal(sys.m)
        if case == 1:
            y[100] = 1e-16  # y below the range
        if case == 2:
            y[::7] = 0.0    # zero y splits exactly
        ex, mag = _exact_t(sys, y, x0)
        g = _aprod2(sys, y, x0, _lib.GSR_PRODUCTS_SPLIT)
        assert np.all(_err(g, ex) <= 30 * U * mag), case


INSTR_ONLY = _lib.GSR_PRODUCTS_MASK | _lib.GSR_SPLIT_APROD2_INSTR


def _instrument_entries(sys):
    """(row, slot) pairs of every instrument, in row order."""
    out = [[] for _ in range(sys.n_instr)]
    for i in range(sys.m):
        for j in range(6):
            out[int(sys.instr[i, j])].append((i, j))
    return out


@pytest.mark.parametrize("products", [INSTR_ONLY, _lib.GSR_PRODUCTS_SPLIT])
def test_split_instrument_sums_exact_under_cancellation(products):
    # aprod 2's instrumental sums: in every instrument the last entry's value
    # cancels the instrument's other products (about 2^41 each), so the
    # exact column sum is a rounding residual; each instrument holds a few
    # hundred entries (the unit's four-entry loop and its tail)
    sys = small(40, 12, 9, obs=9, seed=21)
    rng = np.random.default_rng(21)
    vals = sys.values.copy()
    vals[:, 17:23] = rng.uniform(1.0, 2.0, size=(sys.m, 6)) * 2.0 ** 20
    y = rng.uniform(1.0, 2.0, size=sys.m) * 2.0 ** 20 * np.where(np.arange(sys.m) % 2 == 0, 1, -1)
    for ent in _instrument_entries(sys):
        part = sum(Fraction(float(vals[i, 17 + j])) * Fraction(float(y[i])) for i, j in ent[:-1])
        i, j = ent[-1]
        vals[i, 17 + j] = -float(part / Fraction(float(y[i])))
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x0 = np.zeros(sys.n)
    ex, mag = _exact_t(sys, y, x0)
    exf = np.array([float(e) for e in ex])
    ins = 5 * sys.n_stars + 3 * sys.n_dfa + np.arange(sys.n_instr)
    assert min(len(e) for e in _instrument_entries(sys)) > 128
    assert np.median(mag[ins] / np.maximum(np.abs(exf[ins]), 1e-300)) > 1e6
    g = _aprod2(sys, y, x0, products)
    err = _err(g, ex)
    assert np.all(err[ins] <= 3 * U * np.abs(exf[ins]) + 2.0 ** -60 * mag[ins])
    assert np.all(err <= 30 * U * mag)
    gn = _aprod2(sys, y, x0, _lib.GSR_PRODUCTS_NATIVE)
    errn = _err(gn, ex)
    assert np.all(errn <= 30 * U * mag)
    assert np.max(errn[ins] / np.maximum(np.abs(exf[ins]), 1e-300)) > 1e-12


def test_split_instrument_sums_out_of_range_fall_back():
    # an operand outside the split range sends its instrument unit to native
    # FP64 products; zero values and zero y split exactly
    sys = small(60, 20, 13, obs=12, seed=22)
    rng = np.random.default_rng(23)
    vals = sys.values.copy()
    vals[5, 18] = 1e-13   # instrumental value below the split range
    vals[40, 21] = 5e11   # above it
    vals[41, 17] = 0.0    # zero value
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x0 = rng.standard_normal(sys.n)
    for case in range(3):
        y = rng.standard_normal(sys.m)
        if case == 1:
            y[100] = 1e-16  # y below the range: six units fall back
        if case == 2:
            y[::7] = 0.0    # zero y splits exactly
        ex, mag = _exact_t(sys, y, x0)
        for products in (INSTR_ONLY, _lib.GSR_PRODUCTS_SPLIT):
            g = _aprod2(sys, y, x0, products)
            assert np.all(_err(g, ex) <= 30 * U * mag), (case, products)


ATT = _lib.GSR_PRODUCTS_MASK | _lib.GSR_SPLIT_APROD2_ATT
ATT2 = _lib.GSR_PRODUCTS_MASK | _lib.GSR_SPLIT_APROD2_ATT2
ATT_INSTR = ATT | _lib.GSR_SPLIT_APROD2_INSTR


def _offset_groups(sys):
    """Rows of every attitude offset, in row order."""
    out = {}
    for i in range(sys.m):
        out.setdefault(int(sys.attoff[i]), []).append(i)
    return out


@pytest.mark.parametrize("products,axes", [(ATT, (2,)), (ATT2, (1, 2)), (ATT_INSTR, (2,))])
def test_split_attitude_sums_exact_under_cancellation(products, axes):
    # aprod 2's attitude sums: in every offset the last row's 12 attitude
    # values cancel the offset's other products of the same axis and tap
    # (about 2^40 each), so every partial sum S[o][a][j] of an attitude unit
    # is a rounding residual; an offset holds more than 32 rows (a unit's
    # loop and its tail).  The column a D + k adds the four residuals of
    # offsets k-3..k, so the bound is on their magnitudes.
    sys = small(40, 12, 9, obs=12, seed=31)
    rng = np.random.default_rng(31)
    vals = sys.values.copy()
    vals[:, 5:17] = rng.uniform(1.0, 2.0, size=(sys.m, 12)) * 2.0 ** 20
    y = rng.uniform(1.0, 2.0, size=sys.m) * 2.0 ** 20 * np.where(np.arange(sys.m) % 2 == 0, 1, -1)
    groups = _offset_groups(sys)
    assert min(len(g) for g in groups.values()) > 32
    resid = {}  # exact partial sum of every (offset, tap)
    for o, rows in groups.items():
        last = rows[-1]
        for t in range(12):
            part = sum(Fraction(float(vals[i, 5 + t])) * Fraction(float(y[i])) for i in rows[:-1])
            vals[last, 5 + t] = -float(part / Fraction(float(y[last])))
            resid[o, t] = part + Fraction(float(vals[last, 5 + t])) * Fraction(float(y[last]))
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x0 = np.zeros(sys.n)
    ex, mag = _exact_t(sys, y, x0)
    D, att0 = sys.n_dfa, 5 * sys.n_stars
    rmag = np.zeros(sys.n)  # sum over the column's offsets of |residual partial|
    for (o, t), r in resid.items():
        a, j = divmod(t, 4)
        rmag[att0 + a * D + o + j] += abs(float(r))
    cols = np.array([att0 + a * D + k for a in axes for k in range(D)])
    assert np.median(mag[cols] / np.maximum(rmag[cols], 1e-300)) > 1e6
    g = _aprod2(sys, y, x0, products)
    err = _err(g, ex)
    assert np.all(err[cols] <= 4 * U * rmag[cols] + 2.0 ** -59 * mag[cols])
    assert np.all(err <= 30 * U * mag)
    # native FP64 products lose up to 2^-53 of the magnitudes per product
    gn = _aprod2(sys, y, x0, _lib.GSR_PRODUCTS_NATIVE)
    errn = _err(gn, ex)
    assert np.all(errn <= 30 * U * mag)
    assert np.max(errn[cols] / np.maximum(rmag[cols], 1e-300)) > 1e-12


@pytest.mark.parametrize("products", [ATT, ATT2])
def test_split_attitude_sums_out_of_range_fall_back(products):
    # an operand outside the split range sends its attitude unit to native
    # FP64 products; zero values and zero y split exactly
    sys = small(60, 20, 13, obs=12, seed=32)
    rng = np.random.default_rng(33)
    vals = sys.values.copy()
    vals[5, 16] = 1e-13   # axis-2 value below the split range
    vals[40, 11] = 5e11   # axis-1 value above it
    vals[41, 14] = 0.0    # zero value
    sys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    x0 = rng.standard_normal(sys.n)
    for case in range(3):
        y = rng.standard_normal(sys.m)
        if case == 1:
            y[100] = 1e-16  # y below the range: its unit falls back
        if case == 2:
            y[::7] = 0.0    # zero y splits exactly
        ex, mag = _exact_t(sys, y, x0)
        g = _aprod2(sys, y, x0, products)
        assert np.all(_err(g, ex) <= 30 * U * mag), case


@pytest.mark.parametrize("products", [ATT, ATT2, ATT_INSTR])
def test_split_attitude_products_and_solve(products):
    # the attitude split forms against the oracle: both products on the tiny
    # and a ragged system, and the whole solve at equal iteration count
    from tests.test_gpu_parity import check_aprods, compare_solve
    for sys in (gen.make("tiny"), small(300, 30, 20, seed=5)):
        check_aprods(sys, 8, products=products, instr_mode=_lib.GSR_INSTR_SORTED)
    compare_solve(gen.make("tiny"), 200, 1e-12, 1e-12, products=products,
                  instr_mode=_lib.GSR_INSTR_SORTED)


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_split_star_pass_every_lane_count(lanes):
    # the split star pass of aprod 2 (explicit GSR_PRODUCTS_SPLIT) with 4 lanes
    # per star (fewer lanes than sums) up to a whole warp per star
    from tests.test_gpu_parity import check_aprods
    check_aprods(gen.make("tiny"), lanes, products=_lib.GSR_PRODUCTS_SPLIT)


def test_product_forms_report_what_runs():
    from paper_2212_11675_gb300.solver import Solver
    tiny = gen.make("tiny")
    with Solver(tiny) as s:  # default: split aprod 1, native aprod 2
        assert s.product_forms() == (True, 0)
    with Solver(tiny, products=ASTRO) as s:  # staged aprod 1: astrometric products too
        assert s.product_forms() == (2, 0)
        s.set_aprod1_staging(False)  # the register form has no astrometric split
        assert s.product_forms() == (1, 0)
    with Solver(tiny, products=_lib.GSR_PRODUCTS_NATIVE) as s:
        assert s.product_forms() == (False, 0)
    with Solver(tiny, products=_lib.GSR_PRODUCTS_SPLIT) as s:
        assert s.product_forms() == (True, 3)
    with Solver(tiny, products=INSTR_ONLY) as s:
        assert s.product_forms() == (False, 2)
    with Solver(tiny, products=_lib.GSR_PRODUCTS_MASK | _lib.GSR_SPLIT_APROD2_STARS) as s:
        assert s.product_forms() == (False, 1)
    with Solver(tiny, products=ATT) as s:
        assert s.product_forms() == (False, 4)
    with Solver(tiny, products=ATT2 | _lib.GSR_SPLIT_APROD1) as s:
        assert s.product_forms() == (True, 8)
    with Solver(tiny, products=ATT_INSTR) as s:
        assert s.product_forms() == (False, 6)
    with Solver(tiny, products=_lib.GSR_PRODUCTS_SPLIT, instr_mode=_lib.GSR_INSTR_SMEM) as s:
        assert s.product_forms() == (True, 0)  # no single-launch aprod 2 on this path
    # more instruments than the split x fits in shared memory: native aprod 1
    with Solver(small(300, 50, 7000, seed=9)) as s:
        assert s.product_forms()[0] == 0
