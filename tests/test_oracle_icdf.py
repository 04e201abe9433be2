"""Pins the oracle's inverse-CDF (ICDF) gaussian and lognormal.

* scipy.special.ndtri (Cephes, an independent implementation of the normal
  quantile) agrees with the oracle's root-finding inverse of Phi;
* the uniform midpoints are exact and symmetric: z(u) = -z(1 - u);
* u = 1/2 + 2^-24 maps to 2^-24 sqrt(2 pi) (first-order Taylor; the cubic
  term is ~1e-22), and no midpoint equals 1/2;
* the outputs follow the normal / lognormal laws (KS) and the ICDF map is
  monotone in the word.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import DIST_GAUSSIAN_ICDF, DIST_LOGNORMAL_ICDF, DT_F32, DT_F64


def _u_f32(w):
    return (2.0 * (w >> 9).astype(np.float64) + 1.0) * 2.0**-24


def _u_f64(wa, wb):
    x = ((wa.astype(np.uint64) << np.uint64(32)) | wb.astype(np.uint64)) >> np.uint64(12)
    return (2.0 * x.astype(np.float64) + 1.0) * 2.0**-53


def test_icdf_f32_matches_scipy_ndtri():
    from scipy.special import ndtri

    rng = np.random.Generator(np.random.PCG64(2))
    w = rng.integers(0, 2**32, 20000, dtype=np.uint64).astype(np.uint32)
    w[:4] = [0, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF]
    z = oracle.transform_words(DIST_GAUSSIAN_ICDF, DT_F32, 0.0, 1.0, w.size, w)
    ref = ndtri(_u_f32(w))
    assert np.max(np.abs(z - ref) / np.maximum(1.0, np.abs(ref))) < 1e-14
    assert abs(z[0] + z[1]) < 1e-15 and z[0] < -5.29 and z[1] > 5.29


def test_icdf_f64_matches_scipy_ndtri_in_the_tails():
    from scipy.special import ndtri

    rng = np.random.Generator(np.random.PCG64(3))
    wa = rng.integers(0, 2**32, 5000, dtype=np.uint64).astype(np.uint32)
    wb = rng.integers(0, 2**32, 5000, dtype=np.uint64).astype(np.uint32)
    wa[:3] = [0, 0xFFFFFFFF, 0]
    wb[:3] = [0, 0xFFFFFFFF, 0x1000]
    w = np.stack([wa, wb], axis=1).reshape(-1)
    z = oracle.transform_words(DIST_GAUSSIAN_ICDF, DT_F64, 0.0, 1.0, wa.size, w)
    ref = ndtri(_u_f64(wa, wb))
    assert np.max(np.abs(z - ref) / np.maximum(1.0, np.abs(ref))) < 1e-14
    assert z[0] < -8.2 and z[1] > 8.2  # u = 2^-53 and 1 - 2^-53


def test_icdf_symmetry_and_center():
    k = np.arange(0, 1 << 23, 997, dtype=np.uint32)
    w = k << np.uint32(9)
    wm = ((np.uint32((1 << 23) - 1) - k) << np.uint32(9)) | np.uint32(0x1FF)
    z = oracle.transform_words(DIST_GAUSSIAN_ICDF, DT_F32, 0.0, 1.0, w.size, w)
    zm = oracle.transform_words(DIST_GAUSSIAN_ICDF, DT_F32, 0.0, 1.0, wm.size, wm)
    assert np.max(np.abs(z + zm)) < 1e-14
    assert np.all(np.diff(z) > 0)  # monotone in the word
    c = oracle.transform_words(DIST_GAUSSIAN_ICDF, DT_F32, 0.0, 1.0, 1,
                               np.array([1 << 31], dtype=np.uint32))[0]
    # absolute precision near u = 1/2 is limited by Phi(z) ~ 1/2 in long double (~3e-20)
    assert abs(c - 2.0**-24 * math.sqrt(2 * math.pi)) < 1e-18


@pytest.mark.parametrize("engine", [oracle.ENGINE_PHILOX, oracle.ENGINE_MRG])
def test_icdf_laws(engine):
    from scipy import stats

    n = 100000
    z = oracle.generate(engine, 2021, 0, DIST_GAUSSIAN_ICDF, DT_F32, 0.0, 1.0, n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    g = oracle.generate(engine, 5, 0, DIST_GAUSSIAN_ICDF, DT_F64, 2.0, 3.0, n)
    assert stats.kstest((g - 2.0) / 3.0, "norm").pvalue > 1e-3
    x = oracle.generate(engine, 9, 0, DIST_LOGNORMAL_ICDF, DT_F32, 0.0, 1.0, n)
    assert np.all(x > 0) and stats.kstest(np.log(x), "norm").pvalue > 1e-3
    assert oracle.words_for(DIST_GAUSSIAN_ICDF, DT_F32, 5) == 5
    assert oracle.words_for(DIST_LOGNORMAL_ICDF, DT_F64, 5) == 10
