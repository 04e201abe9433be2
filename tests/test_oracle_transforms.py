"""Pins the oracle's distribution transforms.

* Word -> uniform conversions are exact by definition: every one of the 2^24
  FP32 values and random FP64 values are compared with exact rational values.
* The range transform of Sec. 4.3 (Listing 2) is checked for its half-open
  interval, its monotonicity, the cases where it is exact by arithmetic
  ([0,1), [-1,1), a + 0), a case where rounding reaches b and the clamp must
  fire, and its error bound against exact rational arithmetic.
* Box-Muller: special values with closed forms, the error of the long double
  evaluation against Python's libm in double, moments and KS tests against
  the normal and lognormal laws (scipy).
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import DIST_BITS, DIST_GAUSSIAN, DIST_LOGNORMAL, DIST_UNIFORM, DT_F32, DT_F64, DT_U32


def test_u01_f32_all_2_24_values_exact():
    k = np.arange(1 << 24, dtype=np.uint32)
    words = (k << 8) | np.uint32(0xA5)  # low byte must not matter
    got = oracle.transform_words(DIST_UNIFORM, DT_F32, 0.0, 1.0, words.size, words)
    expect = np.ldexp(k.astype(np.float64), -24).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), expect.view(np.uint32))
    assert got[0] == 0.0 and got[-1] == np.float32(1 - 2**-24)


def test_u01_f64_exact():
    rng = np.random.Generator(np.random.PCG64(11))
    w = rng.integers(0, 2**32, size=(20000, 2), dtype=np.uint64).astype(np.uint32)
    w[0] = [0, 0]
    w[1] = [0xFFFFFFFF, 0xFFFFFFFF]
    w[2] = [0, 0x7FF]  # below the 11 dropped bits
    got = oracle.transform_words(DIST_UNIFORM, DT_F64, 0.0, 1.0, w.shape[0], w.reshape(-1))
    for (wa, wb), g in zip(w.tolist(), got.tolist()):
        x = ((wa << 32) | wb) >> 11
        assert Fraction(g) == Fraction(x, 2**53)
    assert got[0] == 0.0 and got[1] == 1 - 2**-53 and got[2] == 0.0


def _f32_words(rng, n):
    w = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    w[:4] = [0, 0xFFFFFFFF, 0x80000000, 0x000000FF]
    return w


@pytest.mark.parametrize("a,b", [(0.0, 1.0), (-1.0, 1.0), (2.5, 3.75), (-1e3, 7.0), (1e-3, 2e-3),
                                 (-5.0, -4.0), (0.5, 1.0)])
def test_uniform_f32_interval_and_error_bound(a, b):
    rng = np.random.Generator(np.random.PCG64(3))
    w = _f32_words(rng, 200000)
    r = oracle.transform_words(DIST_UNIFORM, DT_F32, a, b, w.size, w)
    af, bf = np.float32(a), np.float32(b)
    assert np.all(r >= af) and np.all(r < bf)
    # monotone in the word's top 24 bits
    order = np.argsort(w >> 8, kind="stable")
    assert np.all(np.diff(r[order].astype(np.float64)) >= 0)
    # within 1.5 ulp(max(|a|,|b|)) of the exact a + (b - a) u (two roundings)
    u = np.ldexp((w >> 8).astype(np.float64), -24)
    exact = float(af) + (float(bf) - float(af)) * u  # exact in double for these inputs
    ulp = np.spacing(np.float32(max(abs(af), abs(bf))))
    assert np.max(np.abs(r.astype(np.float64) - exact)) <= 1.5 * float(ulp)
    # the word 0 gives a exactly
    assert r[0] == af


def _round_f32(x: Fraction) -> float:
    """x rounded to the nearest float32 (ties to even), exactly (normal range)."""
    if x == 0:
        return 0.0
    e = math.floor(math.log2(abs(x)))
    while Fraction(2) ** e > abs(x):
        e -= 1
    while Fraction(2) ** (e + 1) <= abs(x):
        e += 1
    ulp = Fraction(2) ** (e - 23)
    return float(round(x / ulp) * ulp)


@pytest.mark.parametrize("a,b", [(-1e3, 7.0), (2.5, 3.75), (1e-3, 2e-3), (-5.0, 3.3)])
def test_uniform_f32_two_roundings(a, b):
    """The reading of Listing 2: d = b - a, then RN(d u), then RN(a + that), each
    rounded to float (no fused multiply-add), against exact rational
    arithmetic with explicit round-to-nearest-even; the fused form differs
    from it on some of these inputs, so a contraction would fail here."""
    rng = np.random.Generator(np.random.PCG64(11))
    w = _f32_words(rng, 3000)
    r = oracle.transform_words(DIST_UNIFORM, DT_F32, a, b, w.size, w)
    af, bf = Fraction(float(np.float32(a))), Fraction(float(np.float32(b)))
    d = Fraction(_round_f32(bf - af))
    fused_differs = 0
    for wi, ri in zip(w.tolist(), r.tolist()):
        u = Fraction(wi >> 8, 2**24)
        want = _round_f32(af + Fraction(_round_f32(d * u)))
        if want >= bf:
            continue  # the clamp case is pinned separately
        assert ri == want, (wi, ri, want)
        fused_differs += _round_f32(af + d * u) != want
    assert fused_differs > 0  # the inputs do tell the two readings apart


def test_uniform_f32_exact_cases():
    k = np.arange(0, 1 << 24, 97, dtype=np.uint32)
    w = k << 8
    r01 = oracle.transform_words(DIST_UNIFORM, DT_F32, 0.0, 1.0, w.size, w)
    r11 = oracle.transform_words(DIST_UNIFORM, DT_F32, -1.0, 1.0, w.size, w)
    for kk, x, y in zip(k.tolist(), r01.tolist(), r11.tolist()):
        assert Fraction(x) == Fraction(kk, 2**24)
        assert Fraction(y) == Fraction(2 * kk, 2**24) - 1  # exact: no rounding happens


def test_uniform_f32_clamp_fires():
    """[0.5, 1): 0.5 + 0.5 (1 - 2^-24) = 1 - 2^-25 ties to 1.0 = b."""
    r = oracle.uniform_f32(0xFFFFFF00, 0.5, 1.0)
    assert r == np.float32(1.0 - 2**-24)
    assert r < 1.0


def test_uniform_f64_interval_exact_cases_and_clamp():
    rng = np.random.Generator(np.random.PCG64(5))
    w = rng.integers(0, 2**32, size=(50000, 2), dtype=np.uint64).astype(np.uint32)
    w[0] = [0xFFFFFFFF, 0xFFFFFFFF]
    r = oracle.transform_words(DIST_UNIFORM, DT_F64, -1.0, 1.0, w.shape[0], w.reshape(-1))
    for (wa, wb), g in zip(w[:2000].tolist(), r[:2000].tolist()):
        x = ((wa << 32) | wb) >> 11
        assert Fraction(g) == Fraction(2 * x, 2**53) - 1
    assert np.all(r >= -1.0) and np.all(r < 1.0)
    # 0.5 + 0.5 (1 - 2^-53) = 1 - 2^-54 ties to 1.0 = b: clamped below b
    assert oracle.uniform_f64(0xFFFFFFFF, 0xFFFFFFFF, 0.5, 1.0) == 1.0 - 2**-53
    r2 = oracle.transform_words(DIST_UNIFORM, DT_F64, 10.0, 11.5, w.shape[0], w.reshape(-1))
    assert np.all(r2 >= 10.0) and np.all(r2 < 11.5)


def test_bits_are_the_words():
    w = np.arange(1000, dtype=np.uint32) * np.uint32(2654435761)
    assert np.array_equal(oracle.transform_words(DIST_BITS, DT_U32, 0, 0, w.size, w), w)


def _bm_pair_f32(w0, w1, mean=0.0, sd=1.0):
    return oracle.transform_words(DIST_GAUSSIAN, DT_F32, mean, sd, 2,
                                  np.array([w0, w1], dtype=np.uint32))


def test_box_muller_f32_special_values():
    # u1 = 1 -> rho = 0
    z = _bm_pair_f32(0xFFFFFFFF, 0x12345678)
    assert z[0] == 0.0 and z[1] == 0.0
    # u2 = 0 -> (rho, 0); u1 = 2^-24 (the smallest) -> rho = sqrt(48 ln 2)
    z = _bm_pair_f32(0x00000000, 0x000000FF)
    rho = math.sqrt(48.0 * math.log(2.0))
    assert abs(z[0] - rho) < 1e-14 and z[1] == 0.0
    # u2 = 1/4 -> (0, rho); u2 = 1/2 -> (-rho, 0)
    k1 = 12345
    u1 = (k1 + 1) / 2**24
    rho = math.sqrt(-2.0 * math.log(u1))
    z = _bm_pair_f32(k1 << 8, (1 << 22) << 8)
    assert abs(z[0]) < 1e-15 and abs(z[1] - rho) < 1e-14
    z = _bm_pair_f32(k1 << 8, (1 << 23) << 8)
    assert abs(z[0] + rho) < 1e-14 and abs(z[1]) < 1e-15
    # mean and stddev enter linearly
    z = _bm_pair_f32(k1 << 8, (1 << 23) << 8, mean=3.0, sd=2.0)
    assert abs(z[0] - (3.0 - 2.0 * rho)) < 1e-13


def test_box_muller_f32_against_double_libm():
    """The long double evaluation agrees with libm in double to ~1e-15."""
    rng = np.random.Generator(np.random.PCG64(9))
    w = rng.integers(0, 2**32, size=4000, dtype=np.uint64).astype(np.uint32)
    z = oracle.transform_words(DIST_GAUSSIAN, DT_F32, 0.0, 1.0, w.size, w)
    for k in range(w.size // 2):
        u1 = ((int(w[2 * k]) >> 8) + 1) / 2**24
        u2 = (int(w[2 * k + 1]) >> 8) / 2**24
        rho = math.sqrt(-2.0 * math.log(u1))
        e0 = rho * math.cos(2 * math.pi * u2)
        e1 = rho * math.sin(2 * math.pi * u2)
        assert abs(z[2 * k] - e0) <= 1e-14 * max(1.0, abs(e0))
        assert abs(z[2 * k + 1] - e1) <= 1e-14 * max(1.0, abs(e1))


def test_box_muller_f64_special_values():
    ones = 0xFFFFFFFF
    z = oracle.transform_words(DIST_GAUSSIAN, DT_F64, 0.0, 1.0, 2,
                               np.array([ones, ones, 0, 0], dtype=np.uint32))
    assert z[0] == 0.0 and z[1] == 0.0
    # u1 = 2^-53 -> rho = sqrt(106 ln 2); u2 = 0
    z = oracle.transform_words(DIST_GAUSSIAN, DT_F64, 0.0, 1.0, 2,
                               np.array([0, 0, 0, 0x7FF], dtype=np.uint32))
    assert abs(z[0] - math.sqrt(106 * math.log(2.0))) < 1e-14 and z[1] == 0.0
    # u2 = 1/4: the FP64 uniform's top bit pattern 0x2000000000000 << 11
    x = 1 << 51
    v = x << 11
    z = oracle.transform_words(DIST_GAUSSIAN, DT_F64, 0.0, 1.0, 2,
                               np.array([0, 0, v >> 32, v & 0xFFFFFFFF], dtype=np.uint32))
    rho = math.sqrt(-2.0 * math.log(2**-53))
    assert abs(z[0]) < 1e-14 and abs(z[1] - rho) < 1e-14


def test_odd_n_consumes_whole_pair():
    w = np.arange(1, 7, dtype=np.uint32) * np.uint32(0x9E3779B9)
    z5 = oracle.transform_words(DIST_GAUSSIAN, DT_F32, 0.0, 1.0, 5, w)
    z6 = oracle.transform_words(DIST_GAUSSIAN, DT_F32, 0.0, 1.0, 6, w)
    assert np.array_equal(z5, z6[:5])
    assert oracle.words_for(DIST_GAUSSIAN, DT_F32, 5) == 6
    assert oracle.words_for(DIST_GAUSSIAN, DT_F64, 5) == 12
    assert oracle.words_for(DIST_LOGNORMAL, DT_F32, 1) == 2
    assert oracle.words_for(DIST_UNIFORM, DT_F64, 5) == 10
    assert oracle.words_for(DIST_UNIFORM, DT_F32, 5) == 5
    assert oracle.words_for(DIST_BITS, DT_U32, 7) == 7
    assert oracle.words_for(DIST_GAUSSIAN, DT_F32, 0) == 0


@pytest.mark.parametrize("engine", [oracle.ENGINE_PHILOX, oracle.ENGINE_MRG])
@pytest.mark.parametrize("dtype", [DT_F32, DT_F64])
def test_gaussian_law(engine, dtype):
    from scipy import stats

    n = 200000
    z = oracle.generate(engine, 2021, 0, DIST_GAUSSIAN, dtype, 0.0, 1.0, n)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    g = oracle.generate(engine, 7, 0, DIST_GAUSSIAN, dtype, 3.0, 0.5, n)
    assert stats.kstest((g - 3.0) / 0.5, "norm").pvalue > 1e-3


@pytest.mark.parametrize("engine", [oracle.ENGINE_PHILOX, oracle.ENGINE_MRG])
def test_lognormal_law(engine):
    from scipy import stats

    n = 200000
    x = oracle.generate(engine, 2021, 0, DIST_LOGNORMAL, DT_F32, 0.0, 1.0, n)
    assert np.all(x > 0)
    assert stats.kstest(np.log(x), "norm").pvalue > 1e-3
    # E x = exp(m + s^2 / 2) for m = 0.25, s = 0.5
    y = oracle.generate(engine, 8, 0, DIST_LOGNORMAL, DT_F32, 0.25, 0.5, n)
    ex = math.exp(0.25 + 0.125)
    sd = math.sqrt((math.exp(0.25) - 1) * math.exp(0.5 + 0.25))
    assert abs(y.mean() - ex) < 5 * sd / math.sqrt(n)


def test_uniform_law():
    from scipy import stats

    u = oracle.generate(oracle.ENGINE_MRG, 2021, 0, DIST_UNIFORM, DT_F64, 0.0, 1.0, 200000)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
