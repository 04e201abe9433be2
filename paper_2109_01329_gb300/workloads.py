"""Seeded synthetic workloads shaped like the paper's (inputs only).

An RNG consumes no data: its inputs are seeds, offsets, sizes and
distribution parameters.  This module produces those, for the tests (which
feed them to both the CUDA library and the oracle) and for bench.py.  It holds
none of the generators' or transforms' arithmetic.

* Single-stream fills: the RNG-burner batches of Sec. 5.1 / Sec. 7 (Philox FP32
  uniform, batch sizes up to 10^8), widened to 10^9 and to both engines and
  all distributions.
* Substreams: 16384 MRG32k3a substreams 2^76 words apart (Philox: 2^40).
* Batched requests and FastCaloSim-shaped demand (Sec. 5.2: three uniforms per
  calorimeter hit, thousands of hits per event) for the batched and served
  forms.
"""

from __future__ import annotations

import math

import numpy as np

# (name, kind, dtype, p0, p1) using the enum values of include/grng.h
BITS, UNIFORM, GAUSSIAN, LOGNORMAL = 0, 1, 2, 3
U32, F32, F64 = 0, 1, 2

SWEEP_DISTS = [
    ("bits_u32", BITS, U32, 0.0, 0.0),
    ("uniform_f32", UNIFORM, F32, 0.0, 1.0),
    ("uniform_f64", UNIFORM, F64, 0.0, 1.0),
    ("gaussian_f32", GAUSSIAN, F32, 0.0, 1.0),
    ("gaussian_f64", GAUSSIAN, F64, 0.0, 1.0),
    ("lognormal_f32", LOGNORMAL, F32, 0.0, 1.0),
]

SWEEP_SIZES = [10**6, 10**7, 10**8, 10**9]
SWEEP_SEED = 2021

# Philox seed 0x12345678, offset 0, 2^20 FP32 uniforms on [0, 1): compared bit for bit
PHILOX_UNIFORM_2POW20 = dict(engine=0, seed=0x12345678, offset=0, n=1 << 20,
                             dist=("uniform_f32", UNIFORM, F32, 0.0, 1.0))

SUBSTREAMS = dict(num_streams=16384, n_per_stream=65536, seed=2021, mrg_stride=1 << 76,
                  philox_stride=1 << 40, dist=("gaussian_f64", GAUSSIAN, F64, 0.0, 1.0))

BATCH_DISTS = [
    ("bits_u32", BITS, U32, 0.0, 0.0),
    ("uniform_f32", UNIFORM, F32, 0.0, 1.0),
    ("gaussian_f32", GAUSSIAN, F32, 0.0, 1.0),
    ("lognormal_f32", LOGNORMAL, F32, 0.0, 1.0),
    ("uniform_f64_pm1", UNIFORM, F64, -1.0, 1.0),
]


def element_size(dtype: int) -> int:
    return 8 if dtype == F64 else 4


def batched_requests(count: int = 4096, seed: int = 2021, lo: int = 64, hi: int = 1 << 20):
    """Request table: engine seeds 1..count, sizes log-uniform in [lo, hi],
    distributions uniform over BATCH_DISTS (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    dists = rng.integers(0, len(BATCH_DISTS), size=count)
    return [dict(seed=i + 1, n=int(sizes[i]), dist=BATCH_DISTS[int(dists[i])])
            for i in range(count)]


def fastcalosim_events(rate_hz: float = 2000.0, duration_s: float = 60.0, seed: int = 2021,
                       mean_hits: float = 8000.0, sigma: float = 0.8, clip=(100, 200000)):
    """Poisson arrivals with lognormal hit counts (arithmetic mean `mean_hits`).

    Returns (arrival_times_s, hits) as numpy arrays.  Each event needs 3h FP32
    uniforms and h FP32 gaussians from its own Philox engine (seed = event id).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_est = int(rate_hz * duration_s * 1.2) + 16
    gaps = rng.exponential(1.0 / rate_hz, size=n_est)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    mu = math.log(mean_hits) - sigma * sigma / 2.0
    hits = np.rint(np.exp(rng.normal(mu, sigma, size=t.size)))
    hits = np.clip(hits, clip[0], clip[1]).astype(np.int64)
    return t, hits


def sample_windows(n: int, count: int = 64, width: int = 4096, seed: int = 7, align: int = 2):
    """Window starts for sampled checks at sizes the oracle cannot cover:
    the head, the tail, every power-of-two boundary and `count` random
    windows; starts are multiples of `align` (whole Box-Muller pairs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    width = min(width, n)
    starts = {0, max(0, n - width)}
    k = 1
    while (1 << k) < n:
        starts.add(max(0, min(n - width, (1 << k) - width // 2)))
        k += 1
    for s in rng.integers(0, max(1, n - width), size=count):
        starts.add(int(s))
    out = sorted({(s // align) * align for s in starts})
    return [(s, min(width, n - s)) for s in out]
