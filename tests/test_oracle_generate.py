"""The oracle's whole path: engine words -> distribution, offsets and continuation."""

import numpy as np
import pytest

import oracle
from oracle import DIST_BITS, DIST_GAUSSIAN, DIST_LOGNORMAL, DIST_UNIFORM, DT_F32, DT_F64, DT_U32

ENGINES = [oracle.ENGINE_PHILOX, oracle.ENGINE_MRG]
DISTS = [(DIST_BITS, DT_U32, 0.0, 0.0), (DIST_UNIFORM, DT_F32, 0.0, 1.0),
         (DIST_UNIFORM, DT_F64, -1.0, 1.0), (DIST_GAUSSIAN, DT_F32, 0.0, 1.0),
         (DIST_GAUSSIAN, DT_F64, 0.0, 1.0), (DIST_LOGNORMAL, DT_F32, 0.0, 1.0),
         (DIST_LOGNORMAL, DT_F64, 0.5, 0.25), (DIST_UNIFORM, DT_F32, 2.0, 5.0)]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("dist", DISTS)
def test_generate_is_transform_of_words(engine, dist):
    d, t, p0, p1 = dist
    for off, n in [(0, 1), (0, 257), (3, 100), (2**40 + 1, 33), (2**76 * 5, 64)]:
        w = oracle.words(engine, 2021, off, oracle.words_for(d, t, n))
        expect = oracle.transform_words(d, t, p0, p1, n, w)
        got = oracle.generate(engine, 2021, off, d, t, p0, p1, n)
        assert np.array_equal(got.view(np.uint8), expect.view(np.uint8))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("dist", DISTS)
def test_continuation(engine, dist):
    """generate(n1) then generate(n2) at the advanced offset == generate(n1 + n2)
    whenever n1 ends on a whole unit (pairs for Box-Muller)."""
    d, t, p0, p1 = dist
    n1, n2 = 10, 23
    a = oracle.generate(engine, 99, 5, d, t, p0, p1, n1)
    b = oracle.generate(engine, 99, 5 + oracle.words_for(d, t, n1), d, t, p0, p1, n2)
    c = oracle.generate(engine, 99, 5, d, t, p0, p1, n1 + n2)
    assert np.array_equal(np.concatenate([a, b]).view(np.uint8), c.view(np.uint8))


def test_empty_and_invalid():
    assert oracle.generate(0, 1, 0, DIST_UNIFORM, DT_F32, 0.0, 1.0, 0).size == 0
    with pytest.raises(ValueError):
        oracle.generate(0, 1, 0, DIST_BITS, DT_F32, 0.0, 1.0, 4)
    with pytest.raises(ValueError):
        oracle.generate(0, 1, 0, DIST_UNIFORM, DT_U32, 0.0, 1.0, 4)
    with pytest.raises(ValueError):
        oracle.generate(5, 1, 0, DIST_UNIFORM, DT_F32, 0.0, 1.0, 4)


def test_philox_uniform_2pow20_head_is_stable():
    """Philox seed 0x12345678, offset 0, 2^20 FP32 uniforms: the first values
    equal the Triton-pinned Philox words through the exact conversion."""
    u = oracle.generate(oracle.ENGINE_PHILOX, 0x12345678, 0, DIST_UNIFORM, DT_F32, 0.0, 1.0,
                        1 << 20)
    w = oracle.words(oracle.ENGINE_PHILOX, 0x12345678, 0, 1 << 20)
    assert np.array_equal(u, np.ldexp((w >> 8).astype(np.float64), -24).astype(np.float32))
    assert u.min() >= 0.0 and u.max() < 1.0


def test_seed_words_reduce_to_single_seeds():
    """One word (MRG) or two words (Philox) equal the single-seed engines;
    Philox counter words equal a word offset of 4 x counter."""
    for seed in [1, 2021, 0xFFFFFFFF, 4294967087 + 3]:
        w32 = seed & 0xFFFFFFFF
        a = oracle.generate_words(oracle.ENGINE_MRG, [w32], 5, DIST_BITS, DT_U32, 0, 0, 50)
        b = oracle.generate(oracle.ENGINE_MRG, w32, 5, DIST_BITS, DT_U32, 0, 0, 50)
        assert np.array_equal(a, b)
    s64 = 0x0123456789ABCDEF
    a = oracle.generate_words(0, [s64 & 0xFFFFFFFF, s64 >> 32], 9, DIST_BITS, DT_U32, 0, 0, 40)
    b = oracle.generate(0, s64, 9, DIST_BITS, DT_U32, 0, 0, 40)
    assert np.array_equal(a, b)
    ctr = [7, 1, 0, 2]
    c = sum(v << (32 * i) for i, v in enumerate(ctr))
    a = oracle.generate_words(0, [1, 2] + ctr, 3, DIST_BITS, DT_U32, 0, 0, 40)
    b = oracle.generate(0, 1 | (2 << 32), (4 * c + 3) % (1 << 128), DIST_BITS, DT_U32, 0, 0, 40)
    assert np.array_equal(a, b)


def test_mrg_seed_words_are_the_state():
    """Six MRG words are the state: the first word follows the recursion from it."""
    M1, M2 = 2**32 - 209, 2**32 - 22853
    w = [11, 22, 33, 44, 55, 66]
    x1 = [w[2], w[1], w[0]]  # (x_{-3}, x_{-2}, x_{-1})
    x2 = [w[5], w[4], w[3]]
    n1 = (1403580 * x1[1] - 810728 * x1[0]) % M1
    n2 = (527612 * x2[2] - 1370589 * x2[0]) % M2
    got = oracle.generate_words(oracle.ENGINE_MRG, w, 0, DIST_BITS, DT_U32, 0, 0, 1)
    assert int(got[0]) == (n1 - n2) % M1
