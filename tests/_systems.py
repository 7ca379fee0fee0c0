"""Edge-case systems for the GPU parity tests (inputs only, no arithmetic)."""
import numpy as np

from paper_2212_11675_gb300 import gen


def drop_stars(sys, empty):
    """Copy of sys in which the stars in `empty` have no observations."""
    counts = np.diff(sys.star_ptr.astype(np.int64))
    keep = np.ones(sys.m, dtype=bool)
    for s in empty:
        keep[sys.star_ptr[s]:sys.star_ptr[s + 1]] = False
        counts[s] = 0
    sp = np.zeros(sys.n_stars + 1, dtype=np.uint32)
    np.cumsum(counts, out=sp[1:])
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sp, sys.attoff[keep].copy(),
                          sys.instr[keep].copy(), sys.values[keep].copy())


def ragged(seed=5, S=257, D=37, I=11):
    """Stars of 0, 1, 2, ... 40 rows; offsets at both ends; instruments at 0 and I-1."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 41, size=S)
    counts[:8] = [1, 0, 2, 33, 0, 1, 64, 7]
    sp = np.zeros(S + 1, dtype=np.uint32)
    np.cumsum(counts, out=sp[1:])
    m = int(sp[-1])
    attoff = rng.integers(0, D - 3, size=m).astype(np.uint32)
    attoff[0], attoff[-1] = 0, D - 4
    instr = np.stack([rng.permutation(I)[:6] for _ in range(m)]).astype(np.uint16)
    instr[0, 0], instr[-1, 5] = 0, I - 1
    values = rng.standard_normal((m, 24))
    return gen.GaiaSystem(S, D, I, sp, attoff, instr, values)


def empty_run(seed=6, run=70000, D=21, I=9):
    """A few stars, then `run` empty stars inside one 32-row tile, then a few
    more: the star of a row is more than 65535 stars past its tile's first."""
    rng = np.random.default_rng(seed)
    counts = np.zeros(run + 6, dtype=np.int64)
    counts[:3] = [5, 3, 2]          # rows 0..9
    counts[3 + run:] = [4, 11, 6]   # rows 10..30, same tile as rows 0..9
    S = len(counts)
    sp = np.zeros(S + 1, dtype=np.uint32)
    np.cumsum(counts, out=sp[1:])
    m = int(sp[-1])
    attoff = rng.integers(0, D - 3, size=m).astype(np.uint32)
    instr = np.stack([rng.permutation(I)[:6] for _ in range(m)]).astype(np.uint16)
    values = rng.standard_normal((m, 24))
    return gen.GaiaSystem(S, D, I, sp, attoff, instr, values)
