"""Row-block sharding of the Gaia system (paper §4, data distribution, Fig. 2).

The rows are cut into P contiguous blocks of whole stars.  Block p holds the
rows of stars s_p .. s_{p+1}-1 and is itself a Gaia system: its stars are
renumbered from 0, and its unknowns are the astrometric columns of its own
stars followed by all 3 D + I + 1 attitude, instrumental and global unknowns,
which every block carries (they are replicated).  Then

  aprod 1:  the rows of block p are y_p += A_p x_p, where x_p is the block's
            astrometric slice of x and the replicated part: no exchange;
  aprod 2:  A_p^T y_p gives the astrometric columns of block p's stars
            (disjoint across blocks) and a partial sum of the replicated
            columns; the partials are summed over the blocks (the reduction
            after aprod 2 in the paper's multi-process scheme).

ShardedProducts runs all blocks on one GPU (one library handle per block) and
sums the replicated partials block after block in a fixed order with the
library's gsr_vector_add kernel.  RankShard is the multi-process form: one
block per rank, the replicated partials summed by torch.distributed's
all_reduce (NCCL between GPUs); its exchange logic is backend-agnostic so it
can be exercised on CPU ranks over gloo.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import gen
from ._lib import check, lib

N_ASTRO = gen.N_ASTRO


def star_blocks(star_ptr, parts: int) -> np.ndarray:
    """Star boundaries b[0] = 0 <= ... <= b[parts] = S of `parts` contiguous
    blocks of whole stars with about m / parts rows each (a block may be
    empty when a single star holds more rows than m / parts)."""
    sp = np.asarray(star_ptr, dtype=np.int64)
    S, m = len(sp) - 1, int(sp[-1])
    if parts < 1:
        raise ValueError("parts must be >= 1")
    b = [0]
    for p in range(1, parts):
        target = (m * p + parts // 2) // parts
        s = int(np.searchsorted(sp, target, side="left"))  # first star starting at or after target
        b.append(min(max(s, b[-1]), S))
    b.append(S)
    return np.array(b, dtype=np.int64)


@dataclass(frozen=True)
class Shard:
    """Block p of a sharded system: stars [s0, s1), rows [r0, r1)."""
    s0: int
    s1: int
    r0: int
    r1: int
    n_stars: int      # S of the whole system
    n_shared: int     # 3 D + I + 1 replicated unknowns

    @property
    def n_astro(self) -> int:
        return N_ASTRO * (self.s1 - self.s0)

    @property
    def n_local(self) -> int:
        return self.n_astro + self.n_shared

    @property
    def astro_slice(self) -> slice:
        """The block's astrometric unknowns in the global x."""
        return slice(N_ASTRO * self.s0, N_ASTRO * self.s1)

    @property
    def shared_slice(self) -> slice:
        """The replicated unknowns in the global x."""
        g0 = N_ASTRO * self.n_stars
        return slice(g0, g0 + self.n_shared)

    def local_system(self, sys: gen.GaiaSystem) -> gen.GaiaSystem:
        """The block as a Gaia system of its own (host arrays)."""
        sp = np.asarray(sys.star_ptr, dtype=np.int64)[self.s0:self.s1 + 1] - self.r0
        return gen.GaiaSystem(self.s1 - self.s0, sys.n_dfa, sys.n_instr, sp.astype(np.uint32),
                              np.ascontiguousarray(sys.attoff[self.r0:self.r1]),
                              np.ascontiguousarray(sys.instr[self.r0:self.r1]),
                              np.ascontiguousarray(sys.values[self.r0:self.r1]))

    def local_x(self, x):
        """x_p = [astrometric slice of this block | replicated part] (a copy)."""
        if isinstance(x, np.ndarray):
            return np.concatenate([x[self.astro_slice], x[self.shared_slice]])
        import torch
        return torch.cat([x[self.astro_slice], x[self.shared_slice]])


def make_shards(sys: gen.GaiaSystem, parts: int) -> list[Shard]:
    sp = np.asarray(sys.star_ptr, dtype=np.int64)
    b = star_blocks(sp, parts)
    n_shared = sys.n - N_ASTRO * sys.n_stars
    return [Shard(int(b[p]), int(b[p + 1]), int(sp[b[p]]), int(sp[b[p + 1]]), sys.n_stars,
                  n_shared) for p in range(parts)]


def vector_add(dst, src, stream=None) -> None:
    """dst += src on the current device (gsr_vector_add; contiguous float64
    CUDA tensors or views)."""
    from .solver import _stream
    if dst.numel() != src.numel():
        raise ValueError("dst and src differ in length")
    check(lib().gsr_vector_add(ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src.data_ptr()),
                               int(dst.numel()), _stream(stream)), "gsr_vector_add")


class ShardedProducts:
    """aprod 1 and aprod 2 of a system split into `parts` star-aligned row
    blocks, all on the current GPU (one library handle per block), with the
    replicated unknowns summed over the blocks in block order."""

    def __init__(self, sys: gen.GaiaSystem, parts: int, **solver_kw):
        from .solver import Solver
        self.m, self.n = sys.m, sys.n
        self.shards = [sh for sh in make_shards(sys, parts)]
        self.solvers = [Solver(sh.local_system(sys), **solver_kw) if sh.r1 > sh.r0 else None
                        for sh in self.shards]

    def close(self):
        for s in self.solvers:
            if s is not None:
                s.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def aprod1(self, x, y, stream=None):
        """y += A x: each block updates its own rows."""
        for sh, s in zip(self.shards, self.solvers):
            if s is not None:
                s.aprod1(sh.local_x(x), y[sh.r0:sh.r1], stream=stream)
        return y

    def aprod2(self, y, x, stream=None):
        """x += A^T y: the astrometric columns from their own block, the
        replicated ones summed over the blocks in block order."""
        import torch
        for sh, s in zip(self.shards, self.solvers):
            if s is None:
                continue
            part = torch.zeros(sh.n_local, dtype=torch.float64, device=y.device)
            s.aprod2(y[sh.r0:sh.r1], part, stream=stream)
            vector_add(x[sh.astro_slice], part[:sh.n_astro], stream)
            vector_add(x[sh.shared_slice], part[sh.n_astro:], stream)
        return x


class RankShard:
    """One row block per rank of a torch.distributed group: `op` computes the
    block's products (aprod1(x_p, y_p): y_p += A_p x_p; aprod2(y_p, x_p):
    x_p += A_p^T y_p) on local vectors, a library Solver on the rank's GPU.
    x_p holds the block's astrometric unknowns and a copy of the replicated
    ones, kept equal on every rank.  `add(dst, src)` adds local vectors
    (vector_add, the library kernel, by default)."""

    def __init__(self, shard: Shard, op, dist, add=None):
        self.shard, self.op, self.dist = shard, op, dist
        self.add = add if add is not None else vector_add

    def aprod1(self, x_local, y_local):
        """y_p += A_p x_p: no exchange."""
        return self.op.aprod1(x_local, y_local)

    def aprod2(self, y_local, x_local):
        """x_p += A_p^T y_p with the replicated partials summed over the
        ranks (one all-reduce of 3 D + I + 1 values)."""
        import torch
        part = torch.zeros(self.shard.n_local, dtype=torch.float64, device=y_local.device)
        self.op.aprod2(y_local, part)
        self.dist.all_reduce(part[self.shard.n_astro:], op=self.dist.ReduceOp.SUM)
        self.add(x_local, part)
        return x_local
