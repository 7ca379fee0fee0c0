"""The input generator: the PyTorch form draws the same streams as the NumPy form.

Both forms implement SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) and the
recipe of the observation system (rows grouped by star and ordered by time,
attitude offset floor(t (D - 3)), six distinct instruments per row, N(0,1)
values).  Integer draws, orders and indices must be identical; normals may
differ in the last bits of log1p/cos.
"""
import numpy as np
import pytest

from paper_2212_11675_gb300 import gen

torch = pytest.importorskip("torch")


def test_splitmix64_first_outputs():
    # SplitMix64 reference outputs for state 0 (published test values of the
    # generator: the first three outputs for seed 0)
    key = np.uint64(0)
    ctr = np.arange(1, 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        got = gen._mix64(key + ctr * gen.GOLDEN)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("shape,seed", [(gen.SHAPES["tiny"], 2212),
                                        (gen.Shape(3000, 300, 50, obs_per_star=None), 77)])
def test_torch_generator_matches_numpy(shape, seed):
    a = gen.generate(shape, seed)
    b = gen.generate_t(shape, seed, "cpu")
    assert b.m == a.m
    assert np.array_equal(b.star_ptr.numpy(), a.star_ptr)
    assert np.array_equal(b.attoff.numpy(), a.attoff)
    assert np.array_equal(b.instr.numpy(), a.instr)
    assert np.allclose(b.values.numpy(), a.values, rtol=4e-16, atol=4e-15)
    assert np.allclose(gen.x_true_t(b, 5, "cpu").numpy(), gen.x_true(a, 5), rtol=4e-16, atol=4e-15)
    assert np.allclose(gen.noise_t(b, 6, "cpu").numpy(), gen.noise(a, 6), rtol=4e-16, atol=4e-18)


def test_u64_t_bits():
    got = gen.u64_t(9, gen.TAG_VALUE, 123, 1000, "cpu").numpy().view(np.uint64)
    assert np.array_equal(got, gen.u64(9, gen.TAG_VALUE, 123, 1000))
