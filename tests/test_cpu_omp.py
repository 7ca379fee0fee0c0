"""The multi-threaded CPU baseline (OpenMP) against the oracle: the same
PC-LSQR up to the order of its thread sums."""
import numpy as np

import oracle
from paper_2212_11675_gb300 import gen
from tests._dense import small
from tests._systems import ragged


def _check(sys, itn, seed):
    xt = gen.x_true(sys, seed)
    b = oracle.aprod1(sys, xt) + gen.noise(sys, seed + 1)
    r = oracle.pc_lsqr(sys, b, itn, 0.0, 0.0)
    q = oracle.omp_pc_lsqr(sys, b, itn, 0.0, 0.0)
    assert q["itn"] == r["itn"] and q["istop"] == r["istop"]
    assert np.linalg.norm(q["x"] - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])
    assert np.abs(q["se"] - r["se"]).max() <= 1e-8 * r["se"].max()
    for k in ("rnorm", "anorm", "acond", "xnorm", "arnorm", "bnorm"):
        assert abs(q[k] - r[k]) <= 1e-9 * abs(r[k]), k


def test_omp_baseline_matches_oracle_tiny():
    _check(gen.make("tiny"), 40, 3)


def test_omp_baseline_matches_oracle_ragged():
    _check(ragged(), 25, 5)
    _check(small(120, 21, 9, seed=4), 30, 7)


def test_omp_baseline_stops_like_the_oracle():
    sys = small(80, 17, 8, seed=2)
    xt = gen.x_true(sys, 1)
    b = oracle.aprod1(sys, xt)  # consistent: stops on S1
    r = oracle.pc_lsqr(sys, b, 500, 1e-10, 1e-10)
    q = oracle.omp_pc_lsqr(sys, b, 500, 1e-10, 1e-10)
    assert q["istop"] == r["istop"] and abs(q["itn"] - r["itn"]) <= 1
    assert oracle.omp_threads() >= 1
