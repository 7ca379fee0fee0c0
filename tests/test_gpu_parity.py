"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: a product is a sum of FP64 terms whose order differs between the
two sides, so element j may differ by a few units of rounding of sum |terms|;
the bound used is 1e-12 * (|A| |x|)_j (|A|^T |y| for aprod 2), far below any
structural mistake.  Solutions are compared at equal iteration counts to
1e-9 relative (norm-wise, and element-wise against the solution's scale).
"""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import _lib, gen
from tests._dense import small
from tests._systems import drop_stars, empty_run, ragged

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _abs_sys(sys):
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                          sys.instr, np.abs(sys.values))


def _solver(sys, **kw):
    from paper_2212_11675_gb300.solver import Solver
    return Solver(sys, **kw)


def check_aprods(sys, lanes=0, seed=0, **kw):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(sys.n)
    y = rng.standard_normal(sys.m)
    y0 = rng.standard_normal(sys.m)
    x0 = rng.standard_normal(sys.n)
    ref1 = oracle.aprod1(sys, x, y0)
    ref2 = oracle.aprod2(sys, y, x0)
    asys = _abs_sys(sys)
    bound1 = 1e-12 * (oracle.aprod1(asys, np.abs(x)) + np.abs(y0)) + 1e-300
    bound2 = 1e-12 * (oracle.aprod2(asys, np.abs(y)) + np.abs(x0)) + 1e-300
    with _solver(sys, lanes_per_star=lanes, **kw) as s:
        yd = torch.tensor(y0, device=DEV)
        s.aprod1(torch.tensor(x, device=DEV), yd)
        xd = torch.tensor(x0, device=DEV)
        s.aprod2(torch.tensor(y, device=DEV), xd)
        torch.cuda.synchronize()
        g1, g2 = yd.cpu().numpy(), xd.cpu().numpy()
    assert np.all(np.abs(g1 - ref1) <= bound1), np.max(np.abs(g1 - ref1) / bound1)
    assert np.all(np.abs(g2 - ref2) <= bound2), np.max(np.abs(g2 - ref2) / bound2)
    assert np.linalg.norm(g1 - ref1) <= 1e-12 * np.linalg.norm(ref1)
    assert np.linalg.norm(g2 - ref2) <= 1e-12 * np.linalg.norm(ref2)


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_aprod_parity_tiny(lanes):
    check_aprods(gen.make("tiny"), lanes)


def test_aprod_parity_ragged_and_empty_stars():
    sys = ragged()
    assert (np.diff(sys.star_ptr.astype(np.int64)) == 0).any()
    check_aprods(sys, 8)
    check_aprods(drop_stars(gen.make("tiny"), [0, 1, 500, 999]), 16, seed=3)


def test_aprod_parity_long_run_of_empty_stars():
    # more than 65535 empty stars inside one 32-row tile: the stored per-row
    # star delta saturates and the kernels walk on over star_ptr
    sys = empty_run()
    assert sys.m <= 32
    check_aprods(sys, 8)
    with _solver(sys, precision=_lib.GSR_PREC_MIXED) as s:
        x = np.random.default_rng(4).standard_normal(sys.n)
        yd = torch.zeros(sys.m, dtype=torch.float64, device=DEV)
        s.aprod1_f32(torch.tensor(x, device=DEV), yd)
        ref = oracle.aprod1_f32(sys, x)
        absys = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                               sys.instr, np.abs(sys.values))
        bound = 1e-12 * oracle.aprod1_f32(absys, np.abs(x))  # of sum |products|
        assert np.all(np.abs(yd.cpu().numpy() - ref) <= bound)


def test_aprod_parity_instruments_beyond_shared_memory():
    # I above the shared-memory privatisation limit; most instruments have
    # no entry at all (empty segments of the instrument-sorted copy)
    check_aprods(small(300, 50, 7000, seed=9), 8)


@pytest.mark.parametrize("mode", [_lib.GSR_INSTR_SMEM, _lib.GSR_INSTR_REPLICAS,
                                  _lib.GSR_INSTR_SORTED])
@pytest.mark.parametrize("shape", ["tiny", "ragged"])
def test_aprod_parity_instrument_modes(mode, shape):
    sys = gen.make("tiny") if shape == "tiny" else small(411, 37, 11, seed=12)
    rng = np.random.default_rng(8)
    y = rng.standard_normal(sys.m)
    ref = oracle.aprod2(sys, y)
    with _solver(sys, instr_mode=mode) as s:
        xd = torch.zeros(sys.n, dtype=torch.float64, device=DEV)
        s.aprod2(torch.tensor(y, device=DEV), xd)
        g = xd.cpu().numpy()
        # the preconditioner runs through the same instrumental path (squares)
        p = torch.zeros(sys.n, dtype=torch.float64, device=DEV)
        s.precondition(p)
        pg = p.cpu().numpy()
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)
    np.testing.assert_allclose(pg, oracle.precondition(sys)[0], rtol=1e-13)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("lanes", [8, 32])
def test_aprod2_schedules(fused, lanes):
    # aprod 2 in one launch (shared work queue) and as separate passes, on a
    # ragged system; the solve graph is captured again after the switch
    sys = small(411, 37, 11, seed=12)
    rng = np.random.default_rng(21)
    y = rng.standard_normal(sys.m)
    ref = oracle.aprod2(sys, y)
    b = _rhs(sys, 5)
    o = oracle.pc_lsqr(sys, b, 40, 0.0, 0.0)
    with _solver(sys, instr_mode=_lib.GSR_INSTR_SORTED, lanes_per_star=lanes) as s:
        s.set_aprod2_fused(not fused)
        s.set_aprod2_fused(fused)
        for _ in range(2):  # the work counter is reset between launches
            xd = torch.zeros(sys.n, dtype=torch.float64, device=DEV)
            s.aprod2(torch.tensor(y, device=DEV), xd)
            g = xd.cpu().numpy()
            assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)
        x, _, res = s.lsqr_solve(torch.tensor(b, device=DEV), 40, 0.0, 0.0, want_se=False)
    assert res["itn"] == 40
    xo = o["x"]
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)


def test_aprod2_schedule_needs_sorted_path():
    sys = gen.make("tiny")
    with _solver(sys, instr_mode=_lib.GSR_INSTR_SORTED) as s:
        with pytest.raises(_lib.GsrError):
            _lib.check(_lib.lib().gsr_set_aprod2_fused(s.handle, 2), "gsr_set_aprod2_fused")
    with _solver(sys, instr_mode=_lib.GSR_INSTR_SMEM) as s:
        with pytest.raises(_lib.GsrError):
            s.set_aprod2_fused(True)


def test_sorted_instrument_path_is_deterministic():
    # segment sums in a fixed order: repeated products are bitwise identical
    sys = gen.make("tiny")
    rng = np.random.default_rng(3)
    y = torch.tensor(rng.standard_normal(sys.m), device=DEV)
    with _solver(sys, instr_mode=_lib.GSR_INSTR_SORTED) as s:
        outs = []
        for _ in range(3):
            xd = torch.zeros(sys.n, dtype=torch.float64, device=DEV)
            s.aprod2(y, xd)
            outs.append(xd.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_aprod_parity_single_star():
    check_aprods(small(1, 4, 6, obs=45), 32)


def test_adjoint_identity_on_gpu():
    sys = gen.make("tiny")
    rng = np.random.default_rng(2)
    x = torch.tensor(rng.standard_normal(sys.n), device=DEV)
    y = torch.tensor(rng.standard_normal(sys.m), device=DEV)
    with _solver(sys) as s:
        ax = s.aprod1(x, torch.zeros(sys.m, dtype=torch.float64, device=DEV))
        aty = s.aprod2(y, torch.zeros(sys.n, dtype=torch.float64, device=DEV))
        lhs = float(ax @ y)
        rhs = float(x @ aty)
        scale = float(ax.norm() * y.norm())
    assert abs(lhs - rhs) <= 1e-13 * scale


def test_host_pointers_match_device_pointers():
    sys = ragged(seed=8)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(sys.n)
    y0 = rng.standard_normal(sys.m)
    with _solver(sys) as s:
        yh = y0.copy()
        s.aprod1(x, yh)
        yd = torch.tensor(y0, device=DEV)
        s.aprod1(torch.tensor(x, device=DEV), yd)
        np.testing.assert_array_equal(yh, yd.cpu().numpy())


def test_preconditioner_parity():
    for sys in (gen.make("tiny"), ragged(), small(6, 8, 40, obs=3)):
        p_ref = oracle.precondition(sys)[0]
        with _solver(sys) as s:
            p = s.precondition(torch.empty(sys.n, dtype=torch.float64, device=DEV)).cpu().numpy()
        np.testing.assert_allclose(p, p_ref, rtol=1e-13)


def _rhs(sys, seed):
    xt = gen.x_true(sys, seed)
    return oracle.aprod1(sys, xt) + gen.noise(sys, seed + 1)


def oracle_sensitivity(sys, b, itn, trials=3):
    """Relative change of the oracle's outputs when b is perturbed by one unit
    of rounding: after LSQR has converged, var, anorm, acond and arnorm are
    sums over iterations whose vectors are dominated by rounding, so they are
    determined only to this level by the method itself."""
    r0 = oracle.pc_lsqr(sys, b, itn, 0.0, 0.0)
    rng = np.random.default_rng(99)
    sens = {"se": 0.0, "anorm": 0.0, "acond": 0.0, "arnorm": 0.0}
    for _ in range(trials):
        b2 = b * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=b.size))
        r1 = oracle.pc_lsqr(sys, b2, itn, 0.0, 0.0)
        sens["se"] = max(sens["se"], np.max(np.abs(r1["se"] - r0["se"]) / r0["se"].max()))
        for k in ("anorm", "acond", "arnorm"):
            sens[k] = max(sens[k], abs(r1[k] / r0[k] - 1.0))
    return sens


def compare_solve(sys, itmax, atol, btol, seed=1, lanes=0, x_tol=1e-9, early=20, **kw):
    b = _rhs(sys, seed)
    ref = oracle.pc_lsqr(sys, b, itmax, atol, btol)
    ref_early = oracle.pc_lsqr(sys, b, early, 0.0, 0.0)
    with _solver(sys, lanes_per_star=lanes, **kw) as s:
        bd = torch.tensor(b, device=DEV)
        # equal iteration count: stop the GPU where the oracle stopped
        x, se, res = s.lsqr_solve(bd, ref["itn"], 0.0, 0.0)
        x, se = x.cpu().numpy(), se.cpu().numpy()
        xe, see, res_e = s.lsqr_solve(bd, early, 0.0, 0.0)
        xe, see = xe.cpu().numpy(), see.cpu().numpy()
        # and with the tolerances themselves
        _, _, res_tol = s.lsqr_solve(bd, itmax, atol, btol)
    # before convergence every output agrees to the FP64 bar
    assert res_e["itn"] == early
    assert np.linalg.norm(xe - ref_early["x"]) <= x_tol * np.linalg.norm(ref_early["x"])
    np.testing.assert_allclose(see, ref_early["se"], rtol=x_tol)
    for k in ("rnorm", "anorm", "acond", "xnorm", "bnorm", "arnorm"):
        assert res_e[k] == pytest.approx(ref_early[k], rel=x_tol), k
    # at the oracle's stopping iteration
    assert res["itn"] == ref["itn"]
    nx = np.linalg.norm(ref["x"])
    assert np.linalg.norm(x - ref["x"]) <= x_tol * nx
    assert np.max(np.abs(x - ref["x"])) <= x_tol * np.max(np.abs(ref["x"]))
    for k in ("rnorm", "xnorm", "bnorm"):
        assert res[k] == pytest.approx(ref[k], rel=x_tol), k
    sens = oracle_sensitivity(sys, b, ref["itn"])
    tol = {k: max(x_tol, 50.0 * v) for k, v in sens.items()}
    assert np.max(np.abs(se - ref["se"])) <= tol["se"] * ref["se"].max()
    for k in ("anorm", "acond", "arnorm"):
        assert res[k] == pytest.approx(ref[k], rel=tol[k]), k
    assert res_tol["istop"] == ref["istop"]
    assert abs(res_tol["itn"] - ref["itn"]) <= 3
    return res


def test_solve_parity_tiny_config():
    """1,000 stars x 20 observations, D=200, I=60, itmax 200, atol=btol=1e-12."""
    res = compare_solve(gen.make("tiny"), 200, 1e-12, 1e-12)
    assert res["istop"] in (1, 2, 7)


@pytest.mark.parametrize("lanes", [4, 32])
def test_solve_parity_ragged(lanes):
    compare_solve(ragged(seed=11), 300, 1e-10, 1e-10, lanes=lanes)


def test_solve_zero_rhs_gives_zero():
    sys = gen.make("tiny")
    with _solver(sys) as s:
        x, se, res = s.lsqr_solve(torch.zeros(sys.m, dtype=torch.float64, device=DEV), 10)
    assert res["istop"] == 0 and res["itn"] == 0
    assert not x.any().item()


@pytest.mark.parametrize("eager", [False, True])
def test_solve_with_host_buffers(eager):
    sys = ragged(seed=12)
    b = _rhs(sys, 5)
    ref = oracle.pc_lsqr(sys, b, 40, 0.0, 0.0)
    with _solver(sys, eager=eager) as s:
        x, se, res = s.lsqr_solve(b, 40, 0.0, 0.0)
    assert isinstance(x, np.ndarray) and res["itn"] == 40
    assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])
    tol = max(1e-9, 50.0 * oracle_sensitivity(sys, b, 40)["se"])
    assert np.max(np.abs(se - ref["se"])) <= tol * ref["se"].max()


def test_errors_are_reported_not_faulted():
    sys = gen.make("tiny")
    bad = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff.copy(),
                         sys.instr, sys.values)
    bad.attoff[123] = sys.n_dfa - 3           # one knot past the last
    with pytest.raises(_lib.GsrError) as e:
        _solver(bad)
    assert e.value.code == _lib.GSR_ERR_INDEX
    bad = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr.copy(), sys.values)
    bad.instr[7, 2] = sys.n_instr
    with pytest.raises(_lib.GsrError) as e:
        _solver(bad)
    assert e.value.code == _lib.GSR_ERR_INDEX
    vals = sys.values.copy()
    vals[5, 5] = np.nan
    bad = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff,
                         sys.instr, vals)
    with pytest.raises(_lib.GsrError) as e:
        _solver(bad)
    assert e.value.code == _lib.GSR_ERR_NONFINITE
    with _solver(sys) as s:
        b = torch.ones(sys.m, dtype=torch.float64, device=DEV)
        b[17] = float("nan")
        with pytest.raises(_lib.GsrError) as e:
            s.lsqr_solve(b, 10)
        assert e.value.code == _lib.GSR_ERR_NONFINITE
        # the handle stays usable after a reported error
        x, _, res = s.lsqr_solve(torch.ones(sys.m, dtype=torch.float64, device=DEV), 5, 0.0, 0.0)
        assert res["itn"] == 5 and torch.isfinite(x).all().item()


def test_time_iteration_leaves_solves_intact():
    """gsr_time_iteration (the benchmark's in-solve kernel timing) returns
    positive durations, and a solve after it is bit-identical to one before."""
    sys = gen.make("tiny")
    b = _rhs(sys, 3)
    with _solver(sys) as s:
        bd = torch.tensor(b, device=DEV)
        x0 = s.lsqr_solve(bd, 30, 0.0, 0.0)[0].cpu().numpy()
        t = s.time_iteration(bd, iters=5)
        assert set(t) == {"aprod1", "aprod2", "vector_pass"}
        assert all(v > 0.0 for v in t.values())
        x1 = s.lsqr_solve(bd, 30, 0.0, 0.0)[0].cpu().numpy()
    np.testing.assert_array_equal(x0, x1)
