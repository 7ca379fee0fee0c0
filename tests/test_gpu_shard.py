"""Row-block sharded products on one GPU (paper §4, Fig. 2): blocks of whole
stars, one library handle per block, the replicated attitude, instrumental
and global partials of aprod 2 summed block after block with gsr_vector_add.
aprod 1 must equal the unsharded handle's row for row (a row's products do
not depend on the other rows), aprod 2 the unsharded handle and the oracle
within 1e-12 of sum |terms|; the block order fixes the sums, so repeated
calls agree bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2212_11675_gb300 import gen, shard
from tests._systems import drop_stars, ragged

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _abs(sys):
    return gen.GaiaSystem(sys.n_stars, sys.n_dfa, sys.n_instr, sys.star_ptr, sys.attoff, sys.instr,
                          np.abs(sys.values))


@pytest.mark.parametrize("parts", [1, 2, 3, 7])
@pytest.mark.parametrize("which", ["tiny", "ragged", "dropped"])
def test_sharded_products_match_the_whole(parts, which):
    from paper_2212_11675_gb300.solver import Solver
    sys = {"tiny": lambda: gen.make("tiny"), "ragged": lambda: ragged(seed=9),
           "dropped": lambda: drop_stars(gen.make("tiny"), [0, 1, 500, 998, 999])}[which]()
    rng = np.random.default_rng(parts)
    x, y = rng.standard_normal(sys.n), rng.standard_normal(sys.m)
    x0, y0 = rng.standard_normal(sys.n), rng.standard_normal(sys.m)
    xd, yd = torch.tensor(x, device=DEV), torch.tensor(y, device=DEV)
    with Solver(sys) as whole:
        y1w = whole.aprod1(xd, torch.tensor(y0, device=DEV)).cpu().numpy()
        x2w = whole.aprod2(yd, torch.tensor(x0, device=DEV)).cpu().numpy()
    with shard.ShardedProducts(sys, parts) as sp:
        y1 = sp.aprod1(xd, torch.tensor(y0, device=DEV)).cpu().numpy()
        x2 = sp.aprod2(yd, torch.tensor(x0, device=DEV)).cpu().numpy()
        x2b = sp.aprod2(yd, torch.tensor(x0, device=DEV)).cpu().numpy()
    np.testing.assert_array_equal(y1, y1w)
    np.testing.assert_array_equal(x2, x2b)
    scale2 = oracle.aprod2(_abs(sys), np.abs(y)) + np.abs(x0)
    assert np.all(np.abs(x2 - x2w) <= 2e-12 * scale2 + 1e-300)
    assert np.all(np.abs(x2 - oracle.aprod2(sys, y, x0)) <= 1e-12 * scale2 + 1e-300)


def test_sharded_products_medium():
    # the medium workload in 4 blocks: sampled against the oracle on the
    # whole system (astrometric, attitude, instrumental and global columns)
    from paper_2212_11675_gb300.solver import Solver
    sys = gen.make("medium")
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(sys.n), rng.standard_normal(sys.m)
    xd, yd = torch.tensor(x, device=DEV), torch.tensor(y, device=DEV)
    with shard.ShardedProducts(sys, 4, conlim=0.0) as sp:
        y1 = sp.aprod1(xd, torch.zeros(sys.m, dtype=torch.float64, device=DEV)).cpu().numpy()
        x2 = sp.aprod2(yd, torch.zeros(sys.n, dtype=torch.float64, device=DEV)).cpu().numpy()
    with Solver(sys, conlim=0.0) as whole:
        y1w = whole.aprod1(xd, torch.zeros(sys.m, dtype=torch.float64, device=DEV)).cpu().numpy()
    np.testing.assert_array_equal(y1, y1w)
    ref = oracle.aprod2(sys, y)
    scale = oracle.aprod2(_abs(sys), np.abs(y))
    assert np.all(np.abs(x2 - ref) <= 1e-12 * scale + 1e-300)


def test_vector_add_refuses_host_memory():
    from paper_2212_11675_gb300 import _lib
    import ctypes
    L = _lib.lib()
    h = np.zeros(4)
    d = torch.zeros(4, dtype=torch.float64, device=DEV)
    rc = L.gsr_vector_add(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(h.ctypes.data), 4, None)
    assert rc == _lib.GSR_ERR_ARG
    assert L.gsr_vector_add(None, None, 0, None) == _lib.GSR_OK
    assert L.gsr_vector_add(None, None, -1, None) == _lib.GSR_ERR_ARG
