"""Parity at the 1,000,000-star size of the mixed-precision workload (m ~ 7e7,
1.7e9 nonzeros, D = 200,000, I = 20,000) and the 2,000,000-star batched
workload (1.4e8 rows, k = 8), generated on the device.  The oracle
is too slow for whole products here, so it computes outputs one by one: A x on
sampled rows (the oracle run on just those rows), the astrometric columns of
A^T y of sampled stars (the oracle run on those stars' rows, which hold every
nonzero of those columns), the same for the binary32-product operator, plus
the adjoint identity over the whole system.  The shared columns of A^T y are
checked one by one too: an attitude column (axis a, knot k) is touched only
by the rows with attitude offset k-3 .. k, an instrument column only by the
rows that name that instrument, so the oracle run on just those rows (found
on the device) gives the column exactly; the global column, touched by every
row, is the sum of the oracle over consecutive row blocks.  The
mixed-precision solve must reach 1e-9 of the FP64 solution at this size."""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import _lib, gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def large():
    sys = gen.make_t("large", DEV)
    yield sys
    del sys
    torch.cuda.empty_cache()


def _host(sys):
    """star_ptr of a device system on the host."""
    return sys.star_ptr.view(torch.int32).cpu().numpy().astype(np.int64)


def _subsystem(sys, sp, rows):
    """Host copy of the rows `rows` (ascending) with their stars, attitude
    offsets, instruments and values; the column space is the full one."""
    rt = torch.tensor(rows, device=DEV)
    stars = np.searchsorted(sp, rows, side="right") - 1
    counts = np.bincount(stars, minlength=sys.n_stars)
    star_ptr = np.zeros(sys.n_stars + 1, dtype=np.uint32)
    np.cumsum(counts, out=star_ptr[1:])
    attoff = sys.attoff.view(torch.int32)[rt].cpu().numpy().astype(np.uint32)
    instr = sys.instr.view(torch.int16)[rt].cpu().numpy().view(np.uint16)
    values = sys.values[rt].cpu().numpy()
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, star_ptr, attoff,
                          np.ascontiguousarray(instr), values)


def _abs(sub):
    return gen.GaiaSystem(sub.n_stars, sub.n_dfa, sub.n_instr, sub.star_ptr, sub.attoff, sub.instr,
                          np.abs(sub.values))


def _sample(sys, sp, nrows=4000, nstars=300, seed=11):
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(sys.m, size=nrows, replace=False))
    stars = np.sort(rng.choice(sys.n_stars, size=nstars, replace=False))
    star_rows = np.concatenate([np.arange(sp[s], sp[s + 1]) for s in stars])
    return rows, stars, star_rows


def _rows_of_attitude_column(sys, k):
    ao = sys.attoff.view(torch.int32)
    return torch.nonzero((ao >= k - 3) & (ao <= k)).flatten().cpu().numpy()


def _rows_of_instrument(sys, f):
    ins = sys.instr.view(torch.int16).to(torch.int32) & 0xffff
    return torch.nonzero((ins == f).any(dim=1)).flatten().cpu().numpy()


def _column_checks(sys, sp, u, xt, f32, rng):
    """Attitude, instrument and global columns of xt = A^T u against the
    oracle on the rows that touch each column."""
    a2 = oracle.aprod2_f32 if f32 else oracle.aprod2
    S, D, I = sys.n_stars, sys.n_dfa, sys.n_instr
    att0, ins0, glb = 5 * S, 5 * S + 3 * D, 5 * S + 3 * D + I
    cols = []
    picks = [(0, 0), (1, 1), (2, D - 1), (0, D - 2)]
    picks += [(int(rng.integers(3)), int(rng.integers(D))) for _ in range(8)]
    for a, k in picks:
        cols.append((att0 + a * D + k, _rows_of_attitude_column(sys, k)))
    for f in [0, I - 1] + [int(v) for v in rng.integers(0, I, size=6)]:
        cols.append((ins0 + f, _rows_of_instrument(sys, f)))
    got = xt[torch.tensor([c for c, _ in cols], device=DEV)].cpu().numpy()
    for (c, rows), g in zip(cols, got):
        assert rows.size > 0, c
        sub = _subsystem(sys, sp, rows)
        us = u[torch.tensor(rows, device=DEV)].cpu().numpy()
        ref = a2(sub, us)[c]
        assert abs(g - ref) <= 1e-12 * a2(_abs(sub), np.abs(us))[c], c
    # the global column over blocks of rows
    ref = scale = 0.0
    block = 8 << 20
    for r0 in range(0, sys.m, block):
        rows = np.arange(r0, min(sys.m, r0 + block))
        sub = _subsystem(sys, sp, rows)
        us = u[r0:r0 + rows.size].cpu().numpy()
        ref += a2(sub, us)[glb]
        scale += a2(_abs(sub), np.abs(us))[glb]
    assert abs(float(xt[glb]) - ref) <= 1e-12 * scale


@pytest.mark.parametrize("precision", [_lib.GSR_PREC_FP64, _lib.GSR_PREC_MIXED])
def test_large_products_sampled(large, precision):
    from paper_2212_11675_gb300.solver import Solver
    sys = large
    assert 6.5e7 < sys.m < 7.5e7 and sys.n == 5_620_001
    sp = _host(sys)
    rows, stars, star_rows = _sample(sys, sp)
    g = torch.Generator(device=DEV).manual_seed(3)
    x = torch.randn(sys.n, dtype=torch.float64, device=DEV, generator=g)
    u = torch.randn(sys.m, dtype=torch.float64, device=DEV, generator=g)
    f32 = precision == _lib.GSR_PREC_MIXED
    with Solver(sys, conlim=0.0, precision=precision, validate=False) as s:
        y = torch.zeros(sys.m, dtype=torch.float64, device=DEV)
        xt = torch.zeros(sys.n, dtype=torch.float64, device=DEV)
        if f32:
            s.aprod1_f32(x, y)
            s.aprod2_f32(u, xt)
        else:
            s.aprod1(x, y)
            s.aprod2(u, xt)
            # adjoint identity over the whole system
            lhs = float(torch.dot(y, u))
            rhs = float(torch.dot(x, xt))
            assert abs(lhs - rhs) <= 1e-12 * float(torch.linalg.norm(y) * torch.linalg.norm(u))
        y_s = y[torch.tensor(rows, device=DEV)].cpu().numpy()
        cols = (5 * stars[:, None] + np.arange(5)[None, :]).ravel()
        xt_s = xt[torch.tensor(cols, device=DEV)].cpu().numpy()
        _column_checks(sys, sp, u, xt, f32, np.random.default_rng(17))
    xh = x.cpu().numpy()
    sub = _subsystem(sys, sp, rows)
    ref1 = oracle.aprod1_f32(sub, xh) if f32 else oracle.aprod1(sub, xh)
    scale1 = (oracle.aprod1_f32 if f32 else oracle.aprod1)(_abs(sub), np.abs(xh))
    assert np.all(np.abs(y_s - ref1) <= 1e-12 * scale1)
    subs = _subsystem(sys, sp, star_rows)
    us = u[torch.tensor(star_rows, device=DEV)].cpu().numpy()
    ref2 = (oracle.aprod2_f32 if f32 else oracle.aprod2)(subs, us)[cols]
    scale2 = (oracle.aprod2_f32 if f32 else oracle.aprod2)(_abs(subs), np.abs(us))[cols]
    assert np.all(np.abs(xt_s - ref2) <= 1e-12 * scale2)


def test_large_mixed_solve_reaches_fp64_solution(large):
    """The mixed-precision solve (binary32 inner products, FP64 refinement)
    reaches 1e-9 relative error against the FP64 PC-LSQR solution at 1e6
    stars, and its reported rnorm is the FP64 ||b - A x|| of its x."""
    from paper_2212_11675_gb300.solver import Solver
    sys = large
    seed = gen.SEEDS["large"]
    with Solver(sys, conlim=0.0, precision=_lib.GSR_PREC_MIXED, validate=False) as s:
        xt = gen.x_true_t(sys, seed, DEV)
        b = gen.noise_t(sys, seed + 1, DEV)
        s.aprod1(xt, b)
        xr, _, rr = s.lsqr_solve(b, 20000, 1e-15, 1e-15, want_se=False)
        xm, res = s.mixed_solve(b, max_outer=30, max_inner=500, inner_tol=1e-3, atol=1e-10)
        ax = torch.zeros(sys.m, dtype=torch.float64, device=DEV)
        s.aprod1(xm, ax)
        rn = float(torch.linalg.norm(b - ax))
        err = float(torch.linalg.norm(xm - xr) / torch.linalg.norm(xr))
    assert rr["istop"] in (1, 2, 4, 5)
    assert res["converged"] == 1
    assert err <= 1e-9, err
    assert res["rnorm"] == pytest.approx(rn, rel=1e-9)


def test_xlarge_batched_products_sampled():
    # the 2,000,000-star batched workload (1.4e8 rows, k = 8 columns): the
    # skinny products on sampled rows and on the astrometric columns of
    # sampled stars against the oracle's binary32-product operator
    from paper_2212_11675_gb300.solver import Solver
    sys = gen.make_t("xlarge", DEV)
    assert 1.3e8 < sys.m < 1.5e8 and sys.n == 11_240_001
    sp = _host(sys)
    rows, stars, star_rows = _sample(sys, sp, nrows=2000, nstars=150, seed=12)
    k = 8
    g = torch.Generator(device=DEV).manual_seed(4)
    X = torch.randn((k, sys.n), dtype=torch.float64, device=DEV, generator=g)
    Y = torch.randn((k, sys.m), dtype=torch.float64, device=DEV, generator=g)
    cols = (5 * stars[:, None] + np.arange(5)[None, :]).ravel()
    with Solver(sys, conlim=0.0, precision=_lib.GSR_PREC_MIXED, validate=False) as s:
        Q, T = s.batched_products(X, Y)
        Q_s = Q[:, torch.tensor(rows, device=DEV)].cpu().numpy()
        T_s = T[:, torch.tensor(cols, device=DEV)].cpu().numpy()
        del Q, T
    sub, subs = _subsystem(sys, sp, rows), _subsystem(sys, sp, star_rows)
    asub, asubs = _abs(sub), _abs(subs)
    st = torch.tensor(star_rows, device=DEV)
    for c in range(k):
        xh = X[c].cpu().numpy()
        ref1 = oracle.aprod1_f32(sub, xh)
        # Q is rounded to binary32 after the double-float sum: half an ulp more
        half_ulp = 0.5 * np.spacing(np.abs(ref1).astype(np.float32)).astype(np.float64)
        bound1 = 1e-12 * oracle.aprod1_f32(asub, np.abs(xh)) + half_ulp
        assert np.all(np.abs(Q_s[c] - ref1) <= bound1), c
        us = Y[c][st].cpu().numpy()
        ref2 = oracle.aprod2_f32(subs, us)[cols]
        assert np.all(np.abs(T_s[c] - ref2) <= 1e-12 * oracle.aprod2_f32(asubs, np.abs(us))[cols]), c
    del sys, X, Y
    torch.cuda.empty_cache()
