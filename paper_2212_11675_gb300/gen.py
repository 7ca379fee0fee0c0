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


# ---------------------------------------------------------------------------
# The same streams and recipe drawn with PyTorch on any device, for workloads
# too large to generate on the host in reasonable time.  Integer draws,
# uniforms, counts, orders, offsets and instrument indices are bit-identical
# to the NumPy functions above; normals agree to the last bits of the
# platform's log1p/cos.  uint64 arithmetic is carried in int64 tensors
# (two's-complement wrap-around), with right shifts masked to be logical.

def _s64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


_T_GOLDEN, _T_M1, _T_M2 = _s64(int(GOLDEN)), _s64(int(_M1)), _s64(int(_M2))


def _t_shr(z, k: int):
    return (z >> k) & ((1 << (64 - k)) - 1)


def _t_mix64(z):
    z = (z ^ _t_shr(z, 30)) * _T_M1
    z = (z ^ _t_shr(z, 27)) * _T_M2
    return z ^ _t_shr(z, 31)


def u64_t(seed: int, tag: int, start: int, count: int, device):
    """u64() as an int64 tensor holding the same 64 bits."""
    import torch
    key = _s64(int(stream_key(seed, tag)))
    ctr = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return _t_mix64(ctr * _T_GOLDEN + key)


def uniform_t(seed: int, tag: int, start: int, count: int, device):
    import torch
    return _t_shr(u64_t(seed, tag, start, count, device), 11).to(torch.float64) * (2.0 ** -53)


def normal_t(seed: int, tag: int, start: int, count: int, device, chunk: int = 1 << 24):
    import torch
    out = torch.empty(count, dtype=torch.float64, device=device)
    for c0 in range(0, count, chunk):
        c = min(chunk, count - c0)
        uu = uniform_t(seed, tag, 2 * (start + c0), 2 * c, device)
        u1, u2 = uu[0::2], uu[1::2]
        out[c0:c0 + c] = torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)
        del uu, u1, u2
    return out


def generate_t(shape: Shape, seed: int, device, with_values: bool = True) -> GaiaSystem:
    """generate() with PyTorch tensors on `device` (same recipe, same streams)."""
    import torch
    S, D, I = shape.n_stars, shape.n_dfa, shape.n_instr
    if D < N_PARAXIS:
        raise ValueError("need at least 4 attitude knots per axis")
    if I < N_INSTR:
        raise ValueError("need at least 6 instrument unknowns")
    i64 = torch.int64
    if shape.obs_per_star is not None:
        cnt = torch.full((S,), shape.obs_per_star, dtype=i64, device=device)
    else:
        lam, clip = shape.lam, shape.clip
        kmax = int(lam + 40 * math.sqrt(lam) + 40)
        pmf = np.empty(kmax + 1)
        pmf[0] = math.exp(-lam)
        for k in range(1, kmax + 1):
            pmf[k] = pmf[k - 1] * lam / k
        cdf = torch.tensor(np.cumsum(pmf), device=device)
        u = uniform_t(seed, TAG_COUNT, 0, S, device)
        cnt = torch.searchsorted(cdf, u, right=True).clamp(max=kmax).clamp(min=clip).to(i64)
    star_ptr = torch.zeros(S + 1, dtype=i64, device=device)
    torch.cumsum(cnt, 0, out=star_ptr[1:])
    m = int(star_ptr[-1])
    if m >= 2 ** 32:
        raise ValueError("too many rows for 32-bit row indices")
    t = uniform_t(seed, TAG_TIME, 0, m, device)
    star_of_row = torch.repeat_interleave(torch.arange(S, dtype=i64, device=device), cnt)
    order = torch.argsort(t, stable=True)                               # time minor
    order = order[torch.argsort(star_of_row[order], stable=True)]      # star major
    del star_of_row
    t = t[order]
    del order
    attoff = torch.floor(t * (D - 3)).to(i64).clamp(max=D - 4).to(torch.uint32)
    del t
    instr = torch.empty((m, N_INSTR), dtype=i64, device=device)
    u = uniform_t(seed, TAG_INSTR, 0, N_INSTR * m, device).view(m, N_INSTR)
    for j in range(N_INSTR):
        top = I - N_INSTR + j
        tj = (u[:, j] * (top + 1)).to(i64).clamp(max=top)
        if j:
            taken = (instr[:, :j] == tj[:, None]).any(dim=1)
            tj = torch.where(taken, torch.full_like(tj, top), tj)
        instr[:, j] = tj
    del u
    instr = instr.to(torch.uint16)
    values = normal_t(seed, TAG_VALUE, 0, N_PAR * m, device).view(m, N_PAR) if with_values else None
    return GaiaSystem(S, D, I, star_ptr.to(torch.uint32), attoff, instr, values)


def make_t(name: str, device) -> GaiaSystem:
    return generate_t(SHAPES[name], SEEDS[name], device)


def x_true_t(sys: GaiaSystem, seed: int, device):
    return normal_t(seed, TAG_XTRUE, 0, sys.n, device)


def noise_t(sys: GaiaSystem, seed: int, device, sigma: float = 1e-3):
    return sigma * normal_t(seed, TAG_NOISE, 0, sys.m, device)
