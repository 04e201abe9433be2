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


def test_config1_head_is_stable():
    """Philox seed 0x12345678, offset 0, 2^20 FP32 uniforms: the first values
    equal the Triton-pinned Philox words through the exact conversion."""
    u = oracle.generate(oracle.ENGINE_PHILOX, 0x12345678, 0, DIST_UNIFORM, DT_F32, 0.0, 1.0,
                        1 << 20)
    w = oracle.words(oracle.ENGINE_PHILOX, 0x12345678, 0, 1 << 20)
    assert np.array_equal(u, np.ldexp((w >> 8).astype(np.float64), -24).astype(np.float32))
    assert u.min() >= 0.0 and u.max() < 1.0
