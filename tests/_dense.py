"""Dense-matrix helpers for the CPU pins (tiny systems only)."""
import numpy as np

from paper_2212_11675_gb300 import gen


def columns(sys):
    """(m, 24) column index of every stored value, from the paper's §3 layout."""
    S, D, I = sys.n_stars, sys.n_dfa, sys.n_instr
    m = sys.m
    star = np.repeat(np.arange(S), np.diff(sys.star_ptr.astype(np.int64)))
    cols = np.empty((m, 24), dtype=np.int64)
    cols[:, 0:5] = 5 * star[:, None] + np.arange(5)[None, :]
    o = sys.attoff.astype(np.int64)
    for a in range(3):
        cols[:, 5 + 4 * a: 9 + 4 * a] = 5 * S + a * D + o[:, None] + np.arange(4)[None, :]
    cols[:, 17:23] = 5 * S + 3 * D + sys.instr.astype(np.int64)
    cols[:, 23] = 5 * S + 3 * D + I
    return cols


def dense(sys, values=None):
    vals = sys.values if values is None else values
    A = np.zeros((sys.m, sys.n))
    cols = columns(sys)
    rows = np.repeat(np.arange(sys.m), 24)
    np.add.at(A, (rows, cols.ravel()), vals.ravel())
    return A


def small(S, D, I, obs=None, seed=7, lam=20.0, clip=10):
    shape = gen.Shape(S, D, I, obs_per_star=obs, lam=lam, clip=clip)
    return gen.generate(shape, seed)
