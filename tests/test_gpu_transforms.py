"""Transforms on chosen words, through grng_transform_words, vs the oracle.

Random engine words almost never reach the edges of the transforms, so here
the words are built to hit them: u1 = 1 and its neighbours, the smallest u1,
every power-of-two octave of u1, the boundaries of the log reduction table,
every octant boundary and sincos table boundary of u2 (FP64 Box-Muller in
integer fixed point), all 2^24 values of the FP32 uniform, and a sweep of u1 over
its whole FP32 range for the FP32 Box-Muller and lognormal error budgets.
"""

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

M53 = (1 << 53) - 1


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2109_01329_gb300 as grng

    return grng


def _gpu(g, kind, dtype, p0, p1, words: np.ndarray, n: int) -> np.ndarray:
    w = torch.from_numpy(words.astype(np.uint32).view(np.int32)).cuda()
    tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}[dtype]
    out = torch.empty(n, dtype=tdt, device="cuda")
    g.transform_words(g.Distribution(kind, dtype, p0, p1), w, out)
    torch.cuda.synchronize()
    r = out.cpu().numpy()
    return r.view(np.uint32) if dtype == 0 else r


def _check(kind, dtype, got, ref, what):
    if kind in (0, 1):
        gb = got.view(np.uint32 if got.dtype.itemsize == 4 else np.uint64)
        rb = ref.view(np.uint32 if ref.dtype.itemsize == 4 else np.uint64)
        bad = np.nonzero(gb != rb)[0]
        assert bad.size == 0, f"{what}: {bad.size} mismatches at {bad[:5]}"
        return 0.0
    tol = 2e-6 if dtype == 1 else 1e-14
    err = np.abs(got.astype(np.float64) - ref) / np.maximum(1.0, np.abs(ref))
    worst = float(err.max()) if err.size else 0.0
    assert worst <= tol, f"{what}: worst {worst:.3e} > {tol} at {int(np.argmax(err))}"
    return worst


def _x_to_words(x: np.ndarray):
    """Words (w_a, w_b) whose 53-bit FP64 uniform integer is x."""
    x = x.astype(np.uint64)
    return ((x >> np.uint64(21)).astype(np.uint32),
            ((x << np.uint64(11)) & np.uint64(0xFFFFFFFF)).astype(np.uint32))


def _fp64_edge_pairs(seed=1, n_random=100000):
    rng = np.random.Generator(np.random.PCG64(seed))
    e1 = [0, 1, 2, 3, M53, M53 - 1, M53 - 2, M53 - 1000]
    for k in range(54):
        for d in (-2, -1, 0, 1):
            v = (1 << k) + d
            if 0 <= v <= M53:
                e1.append(v)
    for i in range(0, 513):
        for d in (-1, 0, 1):
            m1 = (1 << 53) - i * (1 << 43) + d
            if 1 <= m1 <= (1 << 53):
                e1.append(m1 - 1)
    # u1 just below 1, every octave of delta = 1 - u1 (the relative-accuracy
    # branch of -ln u1 below 2^-10 and its boundary), and u1 around 1/2
    for k in range(0, 53):
        for d in (-1, 0, 1, 3):
            v = M53 - ((1 << k) + d)
            if 0 <= v <= M53:
                e1.append(v)
    for d in range(-40, 41):
        e1.append((1 << 52) - 1 + d)
    e2 = [0, 1, M53, M53 - 1]
    for o in range(9):
        for d in (-2, -1, 0, 1, 2):
            v = o * (1 << 50) + d
            if 0 <= v <= M53:
                e2.append(v)
    for j in range(0, 1025):  # boundaries of the 2 pi / 8192 sincos table
        for d in (-1, 0, 1):
            v = j * (1 << 40) + d
            if 0 <= v <= M53:
                e2.append(v)
    e1 = np.array(sorted(set(e1)), dtype=np.uint64)
    e2 = np.array(sorted(set(e2)), dtype=np.uint64)
    x1 = np.concatenate([rng.integers(0, 1 << 53, n_random, dtype=np.uint64), e1,
                         np.repeat(np.uint64(987654321), e2.size),
                         rng.choice(e1, 20000), ])
    x2 = np.concatenate([rng.integers(0, 1 << 53, n_random, dtype=np.uint64),
                         rng.integers(0, 1 << 53, e1.size, dtype=np.uint64), e2,
                         rng.choice(e2, 20000)])
    a0, a1 = _x_to_words(x1)
    b0, b1 = _x_to_words(x2)
    return np.stack([a0, a1, b0, b1], axis=1).reshape(-1)


@pytest.mark.parametrize("kind,p0,p1", [(2, 0.0, 1.0), (2, -3.0, 0.25), (3, 0.0, 1.0),
                                        (3, 0.5, 0.5)])
def test_fp64_box_muller_edges(g, kind, p0, p1):
    w = _fp64_edge_pairs()
    n = w.size // 2
    got = _gpu(g, kind, 2, p0, p1, w, n)
    ref = oracle.transform_words(kind, 2, p0, p1, n, w)
    _check(kind, 2, got, ref, f"FP64 kind {kind} ({p0}, {p1})")


@pytest.mark.parametrize("m,s", [(0.0, 1.0), (-3.0, 2.0), (650.0, 1.0), (701.0, 0.5),
                                 (-705.0, 2.0), (1.0, 20.0), (1.0, 2.0**-61)])
def test_fp64_lognormal_ranges(g, m, s):
    """The fixed-point lognormal exp(m) 2^(s z log2 e) and its FP64 fallbacks:
    s below 2^-60 sends the whole launch to FP64, outputs below the normal
    range (m = -705) take it one by one; the rest stays in fixed point, also
    where m + s z rounded to a double would lose more than 1e-14 (m = 701)."""
    w = _fp64_edge_pairs(seed=4, n_random=30000)
    n = w.size // 2
    got = _gpu(g, 3, 2, m, s, w, n)
    ref = oracle.transform_words(3, 2, m, s, n, w)
    assert np.all(np.isfinite(got)) and np.all(got >= 0)
    _check(3, 2, got, ref, f"FP64 lognormal ({m}, {s})")


def test_fp64_uniform_edges(g):
    w = _fp64_edge_pairs(seed=2, n_random=50000)
    # the product d u in integers (ordinary ranges, even units) and on the FP64
    # pipe (odd units, and ranges whose products can be subnormal), the clamp as
    # a threshold on the words
    for a, b in [(0.0, 1.0), (-1.0, 1.0), (-0.5, 0.5), (2.0, 5.0), (-1e300, 1e300),
                 (0.25, 0.5), (-4.0, 0.0), (-3.0, 7.5), (0.1, 0.7), (1e15, 1e15 + 3.0),
                 (1.0, 1.0 + 2.0**-40), (3.0, 3.0000000000000004), (-7.25, -7.0),
                 (-1e-300, 1e-300), (0.0, 2.0**-1000), (-2.0**-1060, 2.0**-1060),
                 # b - a with a short significand: the product d u often ties
                 (0.0, 3.0), (-1.0, 2.0), (0.5, 1.25), (1.0, 6.0), (-0.75, 0.625)]:
        # every word pair at an even and at an odd unit index (the transform
        # kernel, like the fills, alternates the integer and the FP64 forms)
        for lead in (0, 1):
            ww = np.concatenate([w[:2 * lead], w])
            nn = ww.size // 2
            got = _gpu(g, 1, 2, a, b, ww, nn)
            ref = oracle.transform_words(1, 2, a, b, nn, ww)
            _check(1, 2, got, ref, f"FP64 uniform [{a}, {b}) lead {lead}")
            assert np.all(got >= a) and np.all(got < b)


def test_fp32_uniform_all_2_24(g):
    k = np.arange(1 << 24, dtype=np.uint32)
    w = (k << np.uint32(8)) | np.uint32(0x5A)
    for a, b in [(0.0, 1.0), (-1.0, 1.0), (0.5, 1.0), (-2.5, 7.0), (1e-3, 2e-3)]:
        got = _gpu(g, 1, 1, a, b, w, w.size)
        ref = oracle.transform_words(1, 1, a, b, w.size, w)
        _check(1, 1, got, ref, f"FP32 uniform [{a}, {b})")


@pytest.mark.parametrize("kind", [2, 3])
def test_fp32_box_muller_u1_sweep(g, kind):
    """Every 16th u1 over its whole range (2^20 values), random u2, plus the u2
    octant points: the FP32 error budget is met everywhere."""
    rng = np.random.Generator(np.random.PCG64(11))
    k1 = np.arange(0, 1 << 24, 16, dtype=np.uint32)
    w0 = (k1 << np.uint32(8)) | rng.integers(0, 256, k1.size, dtype=np.uint32)
    w1 = rng.integers(0, 1 << 32, k1.size, dtype=np.uint64).astype(np.uint32)
    quarter = np.array([0, 1 << 21, 1 << 22, 3 << 21, 1 << 23, 5 << 21, 3 << 22, 7 << 21],
                       dtype=np.uint32) << np.uint32(8)
    w1[: 8 * 1024] = np.tile(quarter, 1024)
    w = np.stack([w0, w1], axis=1).reshape(-1)
    n = w.size
    got = _gpu(g, kind, 1, 0.0, 1.0, w, n)
    ref = oracle.transform_words(kind, 1, 0.0, 1.0, n, w)
    worst = _check(kind, 1, got, ref, f"FP32 kind {kind}")
    print(f"FP32 kind {kind}: worst error / max(1,|x|) = {worst:.3e} (tolerance 2e-6)")


@pytest.mark.parametrize("var", [(0, 0, 0.0, 0.0), (1, 1, 0.0, 1.0), (1, 2, 0.0, 1.0),
                                 (2, 1, 1.0, 3.0), (2, 2, 0.0, 1.0), (3, 1, 0.0, 1.0)])
def test_transform_odd_n_and_random(g, var):
    kind, dtype, p0, p1 = var
    rng = np.random.Generator(np.random.PCG64(5))
    for n in (1, 2, 3, 7, 1001):
        nw = oracle.words_for(kind, dtype, n)
        w = rng.integers(0, 1 << 32, nw, dtype=np.uint64).astype(np.uint32)
        got = _gpu(g, kind, dtype, p0, p1, w, n)
        ref = oracle.transform_words(kind, dtype, p0, p1, n, w)
        _check(kind, dtype, got, ref, f"{var} n={n}")


@pytest.mark.parametrize("kind,p0,p1", [(4, 0.0, 1.0), (5, 0.0, 1.0), (4, -1.0, 3.0)])
def test_icdf_f32_tails_and_sweep(g, kind, p0, p1):
    """Every k in both tails (k < 4096 and k > 2^23 - 4096), every k within
    2048 of the centre and of the two points where the kernel switches from
    its central to its tail polynomial (-log2(1 - x^2) = 5 / ln 2 with
    x = 2u - 1), and every 61st k in between: the inverse CDF meets the FP32
    tolerance across (0, 1)."""
    x1 = np.sqrt(1.0 - np.exp(-5.0))
    seams = [int(((1 << 23) * (1.0 + s * x1) - 1.0) / 2.0) for s in (-1.0, 1.0)] + [1 << 22]
    k = np.concatenate([np.arange(0, 4096), np.arange((1 << 23) - 4096, 1 << 23),
                        np.arange(4096, (1 << 23) - 4096, 61)]
                       + [np.arange(c - 2048, c + 2048) for c in seams]).astype(np.uint32)
    w = (k << np.uint32(9)) | np.uint32(0x155)
    got = _gpu(g, kind, 1, p0, p1, w, w.size)
    ref = oracle.transform_words(kind, 1, p0, p1, w.size, w)
    worst = _check(kind, 1, got, ref, f"ICDF FP32 kind {kind}")
    print(f"ICDF FP32 kind {kind}: worst error / max(1,|x|) = {worst:.3e}")


@pytest.mark.parametrize("kind", [3, 5])
@pytest.mark.parametrize("m,s", [(0.0, 1.0), (-2.0, 1.5), (1.0, 0.5), (85.5, 2.0**-30),
                                 (86.5, 2.0**-30), (-85.5, 2.0**-30), (-86.5, 2.0**-30)])
def test_fp32_lognormal_ranges(g, kind, m, s):
    """FP32 lognormal (Box-Muller and inverse CDF) over parameters: the
    library tolerance for moderate m + s z, and with s = 2^-30 (m + s z rounds
    to m exactly in float) a relative bound of 2e-6 for results near the top
    and the bottom of the normal float range."""
    rng = np.random.Generator(np.random.PCG64(21))
    n = 100001
    nw = oracle.words_for(kind, 1, n)
    w = rng.integers(0, 1 << 32, nw, dtype=np.uint64).astype(np.uint32)
    got = _gpu(g, kind, 1, m, s, w, n)
    ref = oracle.transform_words(kind, 1, m, s, n, w)
    if s < 1e-6:
        rel = np.abs(got.astype(np.float64) - ref) / np.abs(ref)
        assert float(rel.max()) <= 2e-6, f"kind {kind} m={m}: worst relative {rel.max():.3e}"
    else:
        _check(kind, 1, got, ref, f"FP32 lognormal kind {kind} m={m} s={s}")


@pytest.mark.parametrize("kind,p0,p1", [(4, 0.0, 1.0), (5, 0.0, 1.0)])
def test_icdf_f32_all_2_23(g, kind, p0, p1):
    """All 2^23 FP32 inverse-CDF inputs u = (k + 1/2) 2^-23 (the 9 low word
    bits, which the method drops, vary with k) against the oracle, computed
    in chunks on the host's cores."""
    import concurrent.futures as cf
    import os

    k = np.arange(1 << 23, dtype=np.uint32)
    w = (k << np.uint32(9)) | ((k * np.uint32(0x9E3779B1)) >> np.uint32(23))
    got = _gpu(g, kind, 1, p0, p1, w, w.size)
    chunks = np.array_split(w, 64)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        parts = list(ex.map(lambda c: oracle.transform_words(kind, 1, p0, p1, c.size, c), chunks))
    ref = np.concatenate(parts)
    worst = _check(kind, 1, got, ref, f"ICDF FP32 kind {kind}, all inputs")
    print(f"ICDF FP32 kind {kind}, all 2^23 inputs: worst error / max(1,|x|) = {worst:.3e}")


@pytest.mark.parametrize("kind", [4, 5])
def test_icdf_f64_tails(g, kind):
    rng = np.random.Generator(np.random.PCG64(8))
    x = np.concatenate([np.arange(0, 2048, dtype=np.uint64),
                        (1 << 52) - 1 - np.arange(0, 2048, dtype=np.uint64),
                        rng.integers(0, 1 << 52, 20000, dtype=np.uint64)])
    x = x << np.uint64(12)  # the 52-bit integer of the FP64 ICDF uniform
    wa = (x >> np.uint64(32)).astype(np.uint32)
    wb = (x & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    w = np.stack([wa, wb], axis=1).reshape(-1)
    got = _gpu(g, kind, 2, 0.0, 1.0, w, wa.size)
    ref = oracle.transform_words(kind, 2, 0.0, 1.0, wa.size, w)
    _check(kind, 2, got, ref, f"ICDF FP64 kind {kind}")
