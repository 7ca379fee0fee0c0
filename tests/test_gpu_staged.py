"""The staged form of aprod 1 (Alg. 1 with each 32-row tile copied into
shared memory by the bulk-copy engine) against the register form and the
oracle.  Both forms run the same per-row arithmetic, so y = y0 + A x must be
bitwise equal; the LSQR form differs only in the grid's order of the
||U||^2 partial sums, so solves are held to the oracle's 1e-9 bar.  The
bounded waits are exercised by a copy that is announced but never issued:
the launch must end, report GSR_ERR_TIMEOUT, and leave the handle usable."""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import _lib, gen
from tests._dense import small
from tests._systems import drop_stars, empty_run, ragged

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _solver(sys, **kw):
    from paper_2212_11675_gb300.solver import Solver
    return Solver(sys, **kw)


def _bound(sys, x, y0):
    a = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                       sys.instr, np.abs(sys.values))
    return 1e-12 * (oracle.aprod1(a, np.abs(x)) + np.abs(y0)) + 1e-300


def _both_forms(sys, x, y0):
    with _solver(sys) as s:
        out = []
        assert s.aprod1_staging()  # the default where it applies
        for staged in (False, True):
            s.set_aprod1_staging(staged)
            assert s.aprod1_staging() == staged
            yd = torch.tensor(y0, device=DEV)
            s.aprod1(torch.tensor(x, device=DEV), yd)
            out.append(yd.cpu().numpy())
        assert s.kernel_status() == _lib.GSR_OK
    return out


def _systems():
    tiny = gen.make("tiny")
    return {
        "tiny": tiny,
        "ragged": ragged(),
        "empty_stars": drop_stars(tiny, [0, 1, 500, 999]),
        "empty_run": empty_run(),
        # 160,087 rows: about 2.7 tiles per warp of the staged grid (the ring
        # of stages is refilled) and a tail of 23 rows
        "multi_tile": small(8000, 500, 200, seed=9),
    }


@pytest.mark.parametrize("name", ["tiny", "ragged", "empty_stars", "empty_run", "multi_tile"])
def test_staged_equals_register_form(name):
    sys = _systems()[name]
    rng = np.random.default_rng(11)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    reg, stg = _both_forms(sys, x, y0)
    assert np.array_equal(reg.view(np.uint64), stg.view(np.uint64))
    ref = oracle.aprod1(sys, x, y0)
    assert np.all(np.abs(stg - ref) <= _bound(sys, x, y0))


def test_staged_rows_outside_split_range():
    # instrumental x below the split range: the rows that use those entries
    # take the native FP64 products in both forms
    sys = gen.make("tiny")
    rng = np.random.default_rng(12)
    x = rng.standard_normal(sys.n)
    ins0 = 5 * sys.n_stars + 3 * sys.n_dfa
    x[ins0 + 3] = 1e-12
    x[ins0 + 17] = -3e-11
    y0 = np.zeros(sys.m)
    reg, stg = _both_forms(sys, x, y0)
    assert np.array_equal(reg.view(np.uint64), stg.view(np.uint64))
    ref = oracle.aprod1(sys, x, y0)
    assert np.all(np.abs(stg - ref) <= _bound(sys, x, y0))


def test_staged_solve_parity():
    sys = gen.make("tiny")
    xt = gen.x_true(sys, 1)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 2)
    ref = oracle.pc_lsqr(sys, b, 200, 1e-12, 1e-12)
    ref20 = oracle.pc_lsqr(sys, b, 20, 0.0, 0.0)
    with _solver(sys) as s:
        s.set_aprod1_staging(True)
        bd = torch.tensor(b, device=DEV)
        x20, se20, r20 = s.lsqr_solve(bd, 20, 0.0, 0.0)
        x, se, res = s.lsqr_solve(bd, ref["itn"], 0.0, 0.0)
        _, _, rtol_ = s.lsqr_solve(bd, 200, 1e-12, 1e-12)
        x20, se20, x = x20.cpu().numpy(), se20.cpu().numpy(), x.cpu().numpy()
    assert r20["itn"] == 20
    assert np.linalg.norm(x20 - ref20["x"]) <= 1e-9 * np.linalg.norm(ref20["x"])
    np.testing.assert_allclose(se20, ref20["se"], rtol=1e-9)
    for k in ("rnorm", "anorm", "acond", "xnorm", "arnorm"):
        assert r20[k] == pytest.approx(ref20[k], rel=1e-9), k
    assert res["itn"] == ref["itn"]
    assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])
    assert rtol_["istop"] == ref["istop"]
    assert abs(rtol_["itn"] - ref["itn"]) <= 3


def test_staged_mixed_solve_matches_register_form():
    sys = gen.make("tiny")
    b = oracle.aprod1(sys, gen.x_true(sys, 3)) + gen.noise(sys, 4)
    xs = []
    with _solver(sys, precision=_lib.GSR_PREC_MIXED) as s:
        for staged in (False, True):
            s.set_aprod1_staging(staged)
            x, res = s.mixed_solve(torch.tensor(b, device=DEV), 6, 60, 1e-4, 1e-12)
            xs.append(x.cpu().numpy())
    assert np.linalg.norm(xs[1] - xs[0]) <= 1e-12 * np.linalg.norm(xs[0])


def test_expired_wait_is_reported_and_handle_recovers():
    sys = gen.make("tiny")
    rng = np.random.default_rng(13)
    x = rng.standard_normal(sys.n)
    with _solver(sys) as s:
        s.set_aprod1_staging(True)
        assert s.kernel_status() == _lib.GSR_OK
        s.inject_missing_copy(0)  # tile 0's copies are announced, never issued
        yd = torch.zeros(sys.m, dtype=torch.float64, device=DEV)
        s.aprod1(torch.tensor(x, device=DEV), yd)
        assert s.kernel_status() == _lib.GSR_ERR_TIMEOUT
        assert s.kernel_status() == _lib.GSR_OK  # cleared by the read
        with pytest.raises(_lib.GsrError) as e:
            s.lsqr_solve(torch.tensor(rng.standard_normal(sys.m), device=DEV), 2, 0.0, 0.0)
        assert e.value.code == _lib.GSR_ERR_TIMEOUT
        s.inject_missing_copy(-1)
        yd.zero_()
        s.aprod1(torch.tensor(x, device=DEV), yd)
        assert s.kernel_status() == _lib.GSR_OK
        g = yd.cpu().numpy()
    ref = oracle.aprod1(sys, x)
    assert np.all(np.abs(g - ref) <= _bound(sys, x, np.zeros(sys.m)))


def test_staging_needs_split_products():
    sys = gen.make("tiny")
    with _solver(sys, products=_lib.GSR_PRODUCTS_NATIVE) as s:
        with pytest.raises(_lib.GsrError) as e:
            s.set_aprod1_staging(True)
        assert e.value.code == _lib.GSR_ERR_UNSUPPORTED
        assert not s.aprod1_staging()


def test_staged_equals_register_form_medium():
    """The benchmark's size (100,000 stars, ~7e6 rows) in its launch
    configuration: y = A x bitwise equal between the two forms."""
    sys = gen.make("medium")
    rng = np.random.default_rng(14)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    reg, stg = _both_forms(sys, x, y0)
    assert np.array_equal(reg.view(np.uint64), stg.view(np.uint64))


def test_staged_y_not_16_byte_aligned():
    # y at an 8-byte offset cannot be staged by the copy engine: the staged
    # form loads it directly and the result is unchanged
    sys = small(8000, 500, 200, seed=9)
    rng = np.random.default_rng(15)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    out = []
    with _solver(sys) as s:
        for staged in (False, True):
            s.set_aprod1_staging(staged)
            buf = torch.zeros(sys.m + 1, dtype=torch.float64, device=DEV)
            yd = buf[1:]
            assert yd.data_ptr() % 16 == 8
            yd.copy_(torch.tensor(y0, device=DEV))
            s.aprod1(torch.tensor(x, device=DEV), yd)
            out.append(yd.cpu().numpy())
        assert s.kernel_status() == _lib.GSR_OK
    assert np.array_equal(out[0].view(np.uint64), out[1].view(np.uint64))
    ref = oracle.aprod1(sys, x, y0)
    assert np.all(np.abs(out[1] - ref) <= _bound(sys, x, y0))
