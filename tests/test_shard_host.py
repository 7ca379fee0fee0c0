"""Row-block sharding of the products (paper §4, Fig. 2) on the CPU.

The oracle computes each block's products on its own Gaia system; the blocks'
rows must reproduce aprod 1 of the whole system exactly (a row's sum does not
depend on the other rows), and the astrometric columns plus the replicated
partials summed over the blocks must reproduce aprod 2 within 1e-12 of
sum |terms|.  The multi-process form (RankShard) is run over two gloo ranks,
with an oracle-backed block operator supplied by the test."""
import os

import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import gen, shard
from tests._systems import drop_stars, ragged

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _abs(sys):
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff, sys.instr,
                          np.abs(sys.values))


@pytest.mark.parametrize("parts", [1, 2, 3, 8, 40])
def test_star_blocks_are_contiguous_whole_stars(parts):
    sys = ragged(seed=3)
    sp = sys.star_ptr.astype(np.int64)
    shards = shard.make_shards(sys, parts)
    assert len(shards) == parts
    assert shards[0].s0 == 0 and shards[-1].s1 == sys.n_stars
    for a, b in zip(shards, shards[1:]):
        assert a.s1 == b.s0 and a.r1 == b.r0
    for sh in shards:
        assert sh.r0 == sp[sh.s0] and sh.r1 == sp[sh.s1]
        assert sh.n_local == 5 * (sh.s1 - sh.s0) + 3 * sys.n_dfa + sys.n_instr + 1
    # balanced up to the largest star
    biggest = int(np.diff(sp).max())
    for sh in shards:
        assert sh.r1 - sh.r0 <= sys.m / parts + biggest + 1


@pytest.mark.parametrize("parts", [1, 2, 5])
def test_block_products_reproduce_the_whole(parts):
    for sys in (gen.make("tiny"), ragged(seed=4), drop_stars(gen.make("tiny"), [0, 3, 999])):
        rng = np.random.default_rng(parts)
        x, y = rng.standard_normal(sys.n), rng.standard_normal(sys.m)
        ref1, ref2 = oracle.aprod1(sys, x), oracle.aprod2(sys, y)
        scale2 = oracle.aprod2(_abs(sys), np.abs(y))
        y1 = np.zeros(sys.m)
        x2 = np.zeros(sys.n)
        for sh in shard.make_shards(sys, parts):
            if sh.r1 == sh.r0:
                continue
            loc = sh.local_system(sys)
            y1[sh.r0:sh.r1] = oracle.aprod1(loc, sh.local_x(x))
            part = oracle.aprod2(loc, y[sh.r0:sh.r1])
            x2[sh.astro_slice] += part[:sh.n_astro]
            x2[sh.shared_slice] += part[sh.n_astro:]
        np.testing.assert_array_equal(y1, ref1)
        assert np.all(np.abs(x2 - ref2) <= 1e-12 * scale2 + 1e-300)


class _OracleOp:
    """A block operator on CPU tensors backed by the oracle (test only)."""

    def __init__(self, sys):
        self.sys = sys

    def aprod1(self, x, y):
        y.copy_(torch.from_numpy(oracle.aprod1(self.sys, x.numpy(), y.numpy())))
        return y

    def aprod2(self, y, x):
        x.copy_(torch.from_numpy(oracle.aprod2(self.sys, y.numpy(), x.numpy())))
        return x


def _rank_main(rank, world, port, seed):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys = ragged(seed=seed)
        rng = np.random.default_rng(seed)
        x, y = rng.standard_normal(sys.n), rng.standard_normal(sys.m)
        x0 = rng.standard_normal(sys.n)
        sh = shard.make_shards(sys, world)[rank]
        rs = shard.RankShard(sh, _OracleOp(sh.local_system(sys)), dist,
                             add=lambda d, s: d.add_(s))
        # aprod 1: this rank's rows, no exchange
        yl = torch.zeros(sh.r1 - sh.r0, dtype=torch.float64)
        rs.aprod1(torch.from_numpy(sh.local_x(x)), yl)
        np.testing.assert_array_equal(yl.numpy(), oracle.aprod1(sys, x)[sh.r0:sh.r1])
        # aprod 2 accumulating into x0: own astrometric columns, and the
        # replicated ones summed over the ranks by the all-reduce
        xl = torch.from_numpy(sh.local_x(x0))
        rs.aprod2(torch.from_numpy(y[sh.r0:sh.r1].copy()), xl)
        ref = oracle.aprod2(sys, y, x0)
        scale = oracle.aprod2(_abs(sys), np.abs(y)) + np.abs(x0)
        want = sh.local_x(ref)
        tol = 1e-12 * sh.local_x(scale) + 1e-300
        assert np.all(np.abs(xl.numpy() - want) <= tol)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("seed", [5, 6])
def test_rank_shard_exchange_over_two_gloo_ranks(seed):
    import torch.multiprocessing as mp
    port = 29600 + (os.getpid() + seed) % 2000
    mp.spawn(_rank_main, args=(2, port, seed), nprocs=2, join=True)
