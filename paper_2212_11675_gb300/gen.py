"""Seeded synthetic inputs shaped like the Gaia AVU-GSR observation system.

This module only draws random numbers and arranges them; it contains none of
the solver's arithmetic (no products with the matrix, no norms, no LSQR).  Both
the CPU oracle and the CUDA path are fed from here.

Structure (paper §3, "Coefficient matrix structure"):
  * every row is one observation of one star and has 24 nonzeros:
    5 astrometric (the star's own 5 columns: parallax, alpha, delta, mu_alpha,
    mu_delta), 12 attitude (3 axes x 4 consecutive B-spline coefficients,
    axis blocks N_DFA columns apart), 6 instrumental (no fixed pattern) and 1
    global (the PPN gamma);
  * rows are grouped by star (the astrometric block-diagonal) and, inside a
    star, ordered by observation time.

The paper's data are confidential, so the value distribution (N(0,1)), the
observation counts and the time law are stand-ins; the recipe is:
  * times t ~ U[0,1), attitude knot offset o = floor(t * (D - 3)), so the four
    knots o..o+3 of every axis stay inside [0, D);
  * 6 instrument indices per row drawn uniformly without replacement from
    [0, I) (Floyd's sampling algorithm);
  * observations per star: a constant, or max(Poisson(lam), clip);
  * values, x_true ~ N(0,1); noise ~ N(0, sigma).

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
element k of stream (seed, tag) is mix64(key + (k + 1) * GOLDEN) with
key = mix64(seed * 0x100000001b3 + tag).  Uniforms take the top 53 bits;
normals use the Box-Muller transform.  Being counter-based, any slice of any
stream can be regenerated independently (and on a device).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags: one independent stream per purpose
TAG_COUNT, TAG_TIME, TAG_INSTR, TAG_VALUE, TAG_XTRUE, TAG_NOISE = 1, 2, 3, 4, 5, 6

N_ASTRO, N_ATT, N_INSTR, N_GLOB, N_PAR = 5, 12, 6, 1, 24
N_AXES, N_PARAXIS = 3, 4


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.uint64(0x100000001B3) + np.uint64(tag)
    return _mix64(np.asarray(k, dtype=np.uint64))[()]


def u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Elements start .. start+count-1 of stream (seed, tag) as uint64."""
    key = stream_key(seed, tag)
    ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + ctr * GOLDEN)


def uniform(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """U[0,1) doubles with 53 random bits."""
    return (u64(seed, tag, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, tag: int, start: int, count: int, chunk: int = 1 << 24) -> np.ndarray:
    """N(0,1) doubles; normal k uses uniforms 2k and 2k+1 of the stream (Box-Muller, cosine branch)."""
    out = np.empty(count, dtype=np.float64)
    for c0 in range(0, count, chunk):
        c = min(chunk, count - c0)
        uu = uniform(seed, tag, 2 * (start + c0), 2 * c)
        u1, u2 = uu[0::2], uu[1::2]
        out[c0:c0 + c] = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    return out


def poisson_clipped(u: np.ndarray, lam: float, clip: int) -> np.ndarray:
    """max(Poisson(lam), clip) by inversion of the CDF at the given uniforms."""
    kmax = int(lam + 40 * math.sqrt(lam) + 40)
    pmf = np.empty(kmax + 1)
    pmf[0] = math.exp(-lam)
    for k in range(1, kmax + 1):
        pmf[k] = pmf[k - 1] * lam / k
    cdf = np.cumsum(pmf)
    k = np.searchsorted(cdf, u, side="right")
    return np.maximum(np.minimum(k, kmax), clip).astype(np.int64)


@dataclasses.dataclass
class GaiaSystem:
    """Compressed observation system: only the 24 nonzeros per row plus index maps.

    star_ptr : uint32[S+1]  rows of star s are star_ptr[s] .. star_ptr[s+1]-1
    attoff   : uint32[m]    first attitude knot of the row, in [0, D-4]
    instr    : uint16[m,6]  instrument column indices, each in [0, I)
    values   : float64[m,24] nonzeros in the order astro(5) att(3x4) instr(6) glob(1)
    """
    n_stars: int
    n_dfa: int
    n_instr: int
    star_ptr: np.ndarray
    attoff: np.ndarray
    instr: np.ndarray
    values: np.ndarray

    @property
    def m(self) -> int:
        return int(self.star_ptr[-1])

    @property
    def n(self) -> int:
        return N_ASTRO * self.n_stars + N_AXES * self.n_dfa + self.n_instr + N_GLOB


@dataclasses.dataclass(frozen=True)
class Shape:
    n_stars: int
    n_dfa: int
    n_instr: int
    obs_per_star: int | None = 20   # constant count, or None for max(Poisson(lam), clip)
    lam: float = 70.0
    clip: int = 10


# The five workloads the benchmarks and parity tests use (sizes from the
# method's own scale, shrunk to what one GPU holds).
SHAPES = {
    "tiny": Shape(1_000, 200, 60, obs_per_star=20),
    "medium": Shape(100_000, 20_000, 2_000, obs_per_star=None),
    "large": Shape(1_000_000, 200_000, 20_000, obs_per_star=None),
    "xlarge": Shape(2_000_000, 400_000, 40_000, obs_per_star=None),
}
BASE_SEED = 2212
SEEDS = {"tiny": BASE_SEED + 0, "medium": BASE_SEED + 1, "large": BASE_SEED + 3, "xlarge": BASE_SEED + 4}


def star_counts(shape: Shape, seed: int) -> np.ndarray:
    if shape.obs_per_star is not None:
        return np.full(shape.n_stars, shape.obs_per_star, dtype=np.int64)
    return poisson_clipped(uniform(seed, TAG_COUNT, 0, shape.n_stars), shape.lam, shape.clip)


def instruments(seed: int, m: int, n_instr: int, start_row: int = 0) -> np.ndarray:
    """6 distinct indices per row in [0, n_instr): Floyd's algorithm, one uniform per draw."""
    if n_instr < N_INSTR:
        raise ValueError("need at least 6 instrument unknowns")
    u = uniform(seed, TAG_INSTR, N_INSTR * start_row, N_INSTR * m).reshape(m, N_INSTR)
    out = np.empty((m, N_INSTR), dtype=np.int64)
    for j in range(N_INSTR):
        top = n_instr - N_INSTR + j          # draw from [0, top]
        t = np.minimum((u[:, j] * (top + 1)).astype(np.int64), top)
        if j:
            taken = (out[:, :j] == t[:, None]).any(axis=1)
            t = np.where(taken, top, t)
        out[:, j] = t
    return out.astype(np.uint16)


def generate(shape: Shape, seed: int, with_values: bool = True) -> GaiaSystem:
    """Build the system: rows sorted by star, then by observation time."""
    S, D, I = shape.n_stars, shape.n_dfa, shape.n_instr
    if D < N_PARAXIS:
        raise ValueError("need at least 4 attitude knots per axis")
    cnt = star_counts(shape, seed)
    star_ptr = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(cnt, out=star_ptr[1:])
    m = int(star_ptr[-1])
    if m >= 2 ** 32:
        raise ValueError("too many rows for 32-bit row indices")
    t = uniform(seed, TAG_TIME, 0, m)
    star_of_row = np.repeat(np.arange(S, dtype=np.int64), cnt)
    order = np.lexsort((t, star_of_row))   # star major, time minor
    t = t[order]
    attoff = np.minimum(np.floor(t * (D - 3)).astype(np.int64), D - 4).astype(np.uint32)
    instr = instruments(seed, m, I)
    values = normal(seed, TAG_VALUE, 0, N_PAR * m).reshape(m, N_PAR) if with_values else None
    return GaiaSystem(S, D, I, star_ptr.astype(np.uint32), attoff, instr, values)


def x_true(sys: GaiaSystem, seed: int) -> np.ndarray:
    return normal(seed, TAG_XTRUE, 0, sys.n)


def noise(sys: GaiaSystem, seed: int, sigma: float = 1e-3) -> np.ndarray:
    return sigma * normal(seed, TAG_NOISE, 0, sys.m)


def make(name: str) -> GaiaSystem:
    return generate(SHAPES[name], SEEDS[name])
