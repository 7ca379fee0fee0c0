"""Parity at the full medium size (100,000 stars, ~7e6 rows, D=20,000,
I=2,000) in the launch configuration the benchmark uses: both products in
full against the oracle, and a short LSQR run at equal iteration count."""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    return gen.make("medium")


def test_medium_aprods_full(medium):
    from paper_2212_11675_gb300.solver import Solver
    sys = medium
    assert 6.5e6 < sys.m < 7.5e6 and sys.n == 562_001
    rng = np.random.default_rng(0)
    x = rng.standard_normal(sys.n)
    y = rng.standard_normal(sys.m)
    ref1 = oracle.aprod1(sys, x)
    ref2 = oracle.aprod2(sys, y)
    with Solver(sys, conlim=0.0) as s:
        yd = torch.zeros(sys.m, dtype=torch.float64, device="cuda")
        xd = torch.zeros(sys.n, dtype=torch.float64, device="cuda")
        s.aprod1(torch.tensor(x, device="cuda"), yd)
        s.aprod2(torch.tensor(y, device="cuda"), xd)
        g1, g2 = yd.cpu().numpy(), xd.cpu().numpy()
    assert np.linalg.norm(g1 - ref1) <= 1e-12 * np.linalg.norm(ref1)
    assert np.linalg.norm(g2 - ref2) <= 1e-12 * np.linalg.norm(ref2)
    # element-wise against the scale of the terms
    a = gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff, sys.instr,
                       np.abs(sys.values))
    assert np.all(np.abs(g1 - ref1) <= 1e-12 * oracle.aprod1(a, np.abs(x)))
    assert np.all(np.abs(g2 - ref2) <= 1e-12 * oracle.aprod2(a, np.abs(y)))


def test_medium_solve_short(medium):
    from paper_2212_11675_gb300.solver import Solver
    sys = medium
    xt = gen.x_true(sys, 5)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, 6)
    ref = oracle.pc_lsqr(sys, b, 8, 0.0, 0.0)
    with Solver(sys, conlim=0.0) as s:
        x, se, res = s.lsqr_solve(torch.tensor(b, device="cuda"), 8, 0.0, 0.0)
        x, se = x.cpu().numpy(), se.cpu().numpy()
    assert res["itn"] == ref["itn"] == 8
    assert np.linalg.norm(x - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])
    np.testing.assert_allclose(se, ref["se"], rtol=1e-9)
    for k in ("rnorm", "anorm", "acond", "xnorm", "arnorm"):
        assert res[k] == pytest.approx(ref[k], rel=1e-9), k
