"""The split-product arithmetic of the FP64 row kernels (csrc/gsr_split.cuh),
compiled for the host with g++ and checked against exact rational arithmetic:
split3 is exact and its range test right at the window ends, and sums of
products accumulated with acc3_fma stay within 2^-60 of the sum of their
magnitudes, including sums that cancel to about 2^-50 of it.  The same header
is what the GPU kernels compile (no GPU needed here)."""
import math
import os
import random
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_11675_gb300", "csrc")
EMIN, EMAX = -30, 30


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    d = tmp_path_factory.mktemp("split_host")
    (d / "cuda_runtime.h").write_text("")  # the header's only CUDA include
    exe = d / "split_host"
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-std=c++17", "-I", str(d), "-I", CSRC,
                    "-o", str(exe), os.path.join(ROOT, "tests", "split_host.cpp")],
                   check=True, capture_output=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="".join(lines), capture_output=True, text=True,
                             check=True).stdout
        return out.splitlines()
    return run


def _exp(v):
    return math.frexp(v)[1] - 1


def _split_lines(vals):
    return ["S %s\n" % float(v).hex() for v in vals]


def test_split_is_exact_and_the_range_test_is_right(harness):
    rng = random.Random(1)
    vals = []
    for e in (EMIN - 1, EMIN, EMIN + 1, -1, 0, 1, EMAX - 1, EMAX, EMAX + 1):
        for mant in (1.0, 2.0 - 2.0 ** -52, 1.5, 1 + 2.0 ** -52, 1 + 2.0 ** -23,
                     1 + 2.0 ** -29, 1 + 2.0 ** -46, rng.uniform(1, 2)):
            for sgn in (1.0, -1.0):
                vals.append(sgn * mant * 2.0 ** e)
    vals += [rng.gauss(0, 1) for _ in range(2000)]
    out = harness(_split_lines(vals))
    assert len(out) == len(vals)
    for v, line in zip(vals, out):
        h, m, l, ok = line.split()
        in_range = EMIN <= _exp(v) <= EMAX
        assert int(ok) == int(in_range), v
        if in_range:
            pieces = [float.fromhex(t) for t in (h, m, l)]
            assert sum(Fraction(p) for p in pieces) == Fraction(v), v
            # leading 24 bits, then pieces far below: |m| < 2^-23 |h|, |l| < 2^-46 |h|
            assert abs(pieces[1]) < 2.0 ** -22 * abs(pieces[0])
            assert abs(pieces[2]) < 2.0 ** -45 * abs(pieces[0])


def _acc_cases(rng):
    def rnd(lo=EMIN, hi=EMAX):
        return rng.choice((-1, 1)) * rng.uniform(1, 2) * 2.0 ** rng.randint(lo, hi)
    cases = []
    for n in (1, 2, 7, 24, 100, 300):
        for _ in range(60):
            cases.append([(rnd(), rnd()) for _ in range(n)])
            cases.append([(rng.gauss(0, 1), rng.gauss(0, 1e-3)) for _ in range(n)])
    # cancellation: the last product cancels the others up to its own rounding
    for n in (2, 7, 24, 70):
        for _ in range(80):
            pairs = [(rnd(-8, 8), rnd(-8, 8)) for _ in range(n - 1)]
            part = sum(Fraction(a) * Fraction(x) for a, x in pairs)
            x_last = rnd(-4, 4)
            a_last = -float(part / Fraction(x_last))
            pairs.append((a_last, x_last))
            cases.append(pairs)
    return [c for c in cases if all(EMIN <= _exp(a) <= EMAX and EMIN <= _exp(x) <= EMAX
                                    for a, x in c if a != 0 and x != 0)
            and all(a != 0 and x != 0 for a, x in c)]


def test_accumulated_products_within_two_to_the_minus_60(harness):
    cases = _acc_cases(random.Random(2))
    lines = ["A %d %s\n" % (len(c), " ".join("%s %s" % (a.hex(), x.hex()) for a, x in c))
             for c in cases]
    out = harness(lines)
    assert len(out) == len(cases)
    worst = 0.0
    cancelling = 0
    for c, line in zip(cases, out):
        ok, h, m, l, d0, d1 = line.split()
        assert ok == "1"
        exact = sum(Fraction(a) * Fraction(x) for a, x in c)
        mag = sum(abs(Fraction(a) * Fraction(x)) for a, x in c)
        got3 = sum(Fraction(float.fromhex(t)) for t in (h, m, l))
        got2 = Fraction(float.fromhex(d0)) + Fraction(float.fromhex(d1))
        err = max(abs(got3 - exact), abs(got2 - exact)) / mag
        worst = max(worst, float(err))
        if abs(exact) < mag * 2.0 ** -40:
            cancelling += 1
    assert worst <= 2.0 ** -60, math.log2(worst)
    assert cancelling > 100  # the cancellation cases really cancel


def test_split3z_takes_zero_and_agrees_with_split3(harness):
    """split3z, the value-argument form the instrument units use: a zero of
    either sign splits into zero pieces and counts as in range; every other
    value gives split3's pieces and range verdict."""
    rng = random.Random(3)
    vals = [0.0, -0.0, 1.0, -1.5, 2.0 ** EMIN, 2.0 ** (EMIN - 1), 2.0 ** (EMAX + 1)]
    vals += [rng.gauss(0, 1) * 2.0 ** rng.randint(-40, 40) for _ in range(500)]
    zs = harness(["Z %s\n" % float(v).hex() for v in vals])
    ss = harness(_split_lines(vals))
    for v, z, s in zip(vals, zs, ss):
        if v == 0.0:
            h, m, l, ok = z.split()
            assert float.fromhex(h) == float.fromhex(m) == float.fromhex(l) == 0.0 and ok == "1"
        else:
            assert z == s, v


def test_reduction_of_split_partials_is_exact(harness):
    """The binary32 reduce-scatter of the row kernels: FP64 partial sums split
    by split3z and added with acc3_add come out within two binary64 roundings
    of the exact sum plus 2^-60 of the sum of magnitudes, also when the
    partials cancel to 2^-40 of their size (where binary64 adds lose far
    more)."""
    rng = random.Random(7)
    lines, cases = [], []
    for trial in range(300):
        n = rng.choice([2, 5, 8, 12, 16, 32])
        vals = [rng.gauss(0, 1) * 2.0 ** rng.randint(-20, 20) for _ in range(n)]
        if trial % 3 == 0:  # cancel: the last partial undoes the others but a tiny rest
            s = sum(Fraction(v) for v in vals[:-1])
            vals[-1] = float(-s) + float(s) * 2.0 ** -40 * rng.choice([-1, 1])
        cases.append(vals)
        lines.append("R %d %s\n" % (n, " ".join(float(v).hex() for v in vals)))
    out = harness(lines)
    for vals, line in zip(cases, out):
        ok, got = line.split()
        assert ok == "1"
        exact = sum(Fraction(v) for v in vals)
        mag = sum(abs(v) for v in vals)
        err = abs(Fraction(float.fromhex(got)) - exact)
        assert err <= 2 * 2.0 ** -53 * abs(exact) + 2.0 ** -60 * Fraction(mag), vals


def test_reduction_window_is_exact_at_its_ends(harness):
    """The reductions accept partial sums with exponents in [-70, 120] (they
    are only added, never multiplied): split exactly, summed with acc3_add,
    within two binary64 roundings of the exact sum plus 2^-60 of the sum of
    magnitudes, also under cancellation, at both ends of the window; one
    binade beyond either end is reported out of the window."""
    rng = random.Random(8)
    lines, cases = [], []
    for trial in range(300):
        n = rng.choice([2, 5, 8, 12, 16, 32])
        e = rng.choice([-70, -69, -60, 40, 110, 119]) if trial % 2 else rng.randint(-70, 118)
        vals = [math.ldexp(rng.uniform(1.0, 2.0) * rng.choice([-1, 1]), e - rng.randint(0, 2)
                           if e - 2 >= -70 else e) for _ in range(n)]
        if trial % 3 == 0:
            s = sum(Fraction(v) for v in vals[:-1])
            rest = float(s) * 2.0 ** -30 * rng.choice([-1, 1])
            last = float(-s) + rest
            if last == 0.0 or _exp(abs(last)) < -70:
                last = float(-s)
            vals[-1] = last
        cases.append(vals)
        lines.append("W %d %s\n" % (n, " ".join(float(v).hex() for v in vals)))
    out = harness(lines)
    for vals, line in zip(cases, out):
        ok, got = line.split()
        assert ok == ("1" if all(v == 0.0 or -70 <= _exp(abs(v)) <= 120 for v in vals) else "0")
        if ok != "1":
            continue
        exact = sum(Fraction(v) for v in vals)
        mag = sum(abs(v) for v in vals)
        err = abs(Fraction(float.fromhex(got)) - exact)
        assert err <= 2 * 2.0 ** -53 * abs(exact) + 2.0 ** -60 * Fraction(mag), vals
    out = harness(["W 1 %s\n" % math.ldexp(1.5, e).hex() for e in (-71, -70, 120, 121)])
    assert [o.split()[0] for o in out] == ["0", "1", "1", "0"]
