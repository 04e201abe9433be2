"""CUDA path vs the oracle, element by element, through the C ABI.

Bits and uniform outputs must be bit-exact; gaussian and lognormal outputs
within |gpu - oracle| <= 2e-6 max(1, |x|) (FP32) or 1e-14 max(1, |x|) (FP64),
the tolerances the library states.  Small cases cover every variant at
ragged sizes, word offsets mod 4, misaligned pointers, 2^64 carries and canary
bands; the full-size cases run in the same launch configuration as bench.py
and compare sampled windows the oracle computes at their word offsets.
"""

import numpy as np
import pytest

import oracle
from paper_2109_01329_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ENGINES = [0, 1]
# (name, kind, dtype, p0, p1): every kernel variant of the library
VARIANTS = [
    ("bits", 0, 0, 0.0, 0.0),
    ("u01_f32", 1, 1, 0.0, 1.0),
    ("uni_f32", 1, 1, -2.5, 7.0),
    ("uni_f32_clamp", 1, 1, 0.5, 1.0),
    ("u01_f64", 1, 2, 0.0, 1.0),
    ("aff_f64", 1, 2, -1.0, 1.0),
    ("uni_f64", 1, 2, 2.0, 5.0),
    ("gauss_f32", 2, 1, 0.5, 2.0),
    ("logn_f32", 3, 1, 0.0, 1.0),
    ("gauss_f64", 2, 2, -1.0, 0.5),
    ("gauss_f64_std", 2, 2, 0.0, 1.0),
    ("logn_f64", 3, 2, 0.25, 0.75),
    ("icdf_gauss_f32", 4, 1, 0.5, 2.0),
    ("icdf_logn_f32", 5, 1, 0.0, 1.0),
    ("icdf_gauss_f64", 4, 2, 0.0, 1.0),
    ("icdf_logn_f64", 5, 2, 0.25, 0.5),
]

SENTINEL = 0xA5


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2109_01329_gb300 as grng

    return grng


def _torch_dtype(dtype):
    return {0: torch.int32, 1: torch.float32, 2: torch.float64}[dtype]


def _as_uint_view(a: np.ndarray) -> np.ndarray:
    return a.view(np.uint32) if a.dtype.itemsize == 4 else a.view(np.uint64)


def assert_parity(kind, dtype, got: np.ndarray, ref: np.ndarray, what=""):
    assert got.shape == ref.shape, what
    if kind in (0, 1):
        g_bits = got.view(np.uint32) if dtype in (0, 1) else got.view(np.uint64)
        r_bits = ref.view(np.uint32) if dtype in (0, 1) else ref.view(np.uint64)
        bad = np.nonzero(g_bits != r_bits)[0]
        assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[:5]}: " \
                              f"{got[bad[:5]]} vs {ref[bad[:5]]}"
    else:
        tol = 2e-6 if dtype == 1 else 1e-14
        g64 = got.astype(np.float64)
        err = np.abs(g64 - ref)
        lim = tol * np.maximum(1.0, np.abs(ref))
        bad = np.nonzero(~(err <= lim))[0]
        assert bad.size == 0, f"{what}: {bad.size} outside tolerance, first at {bad[:5]}: " \
                              f"{g64[bad[:5]]} vs {ref[bad[:5]]}"


def _gpu_fill(g, engine_kind, seed, offset, var, n, ptr_off=0, guard=16):
    """Generates into the middle of a sentinel-filled buffer; checks the bands."""
    _, kind, dtype, p0, p1 = var
    es = 8 if dtype == 2 else 4
    total = n + ptr_off + 2 * guard
    raw = torch.full((total * es,), SENTINEL, dtype=torch.uint8, device="cuda")
    buf = raw.view(_torch_dtype(dtype))
    out = buf[guard + ptr_off: guard + ptr_off + n]
    e = g.Engine(engine_kind, seed, offset)
    g.generate(g.Distribution(kind, dtype, p0, p1), e, out, n=n)
    torch.cuda.synchronize()
    host = raw.cpu().numpy()
    lo = (guard + ptr_off) * es
    hi = lo + n * es
    assert np.all(host[:lo] == SENTINEL) and np.all(host[hi:] == SENTINEL), "canary band written"
    assert e.offset == (offset + oracle.words_for(kind, dtype, n)) % (1 << 128)
    vals = host[lo:hi].view(np.uint32 if dtype == 0 else (np.float32 if dtype == 1 else np.float64))
    return vals.copy()


def _ref(engine_kind, seed, offset, var, n):
    _, kind, dtype, p0, p1 = var
    return oracle.generate(engine_kind, seed, offset, kind, dtype, p0, p1, n)


SMALL_CASES = [
    # (n, word offset, pointer element offset)
    (1, 0, 0), (2, 0, 1), (3, 1, 0), (5, 2, 3), (7, 3, 2), (64, 0, 0), (1000, 5, 1),
    (4099, 0, 0), (4099, 2, 2), (70001, 3, 1), (262147, 0, 0), (33, (1 << 34) - 7, 0),
    (101, (1 << 64) - 9, 3), (97, (1 << 76) * 3 + 1, 1), (50, (1 << 128) - 30, 0),
    (1001, 2, 1), (65537, 4, 3), (4133, (1 << 66) - 4 * 517 + 2, 1),
]


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("var", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_small_cases_all_variants(g, engine_kind, var):
    for n, off, pofs in SMALL_CASES:
        got = _gpu_fill(g, engine_kind, 2021, off, var, n, ptr_off=pofs)
        ref = _ref(engine_kind, 2021, off, var, n)
        assert_parity(var[1], var[2], got, ref, f"{var[0]} n={n} off={off} ptr+{pofs}")


@pytest.mark.parametrize("ph", [1, 2, 3])
@pytest.mark.parametrize("var", VARIANTS[:3], ids=[v[0] for v in VARIANTS[:3]])
def test_philox_one_word_fills_at_each_word_phase(g, ph, var):
    """Philox fills of one word per output (bits, FP32 uniforms) whose groups
    start at word phase 1, 2 or 3 of a counter block (loops of their own per
    phase): a long fill, at an aligned and a misaligned pointer, equals the
    aligned fill moved by the offset, and a fill across the 2^64 carry of the
    block counter equals the oracle."""
    n = (1 << 22) + 3
    ref = _gpu_fill(g, 0, 2021, 0, var, n + 8)
    for pofs in (0, 1, 3):
        off = (ph + pofs) % 4 + 4  # the groups' word phase is off - pofs mod 4
        got = _gpu_fill(g, 0, 2021, off, var, n, ptr_off=pofs)
        bad = np.nonzero(_as_uint_view(got) != _as_uint_view(ref[off:off + n]))[0]
        assert bad.size == 0, f"phase {ph} ptr+{pofs}: {bad.size} differ, first at {bad[:5]}"
    off = (1 << 66) - 4 * 1000 + ph
    got = _gpu_fill(g, 0, 7, off, var, 100003)
    assert_parity(var[1], var[2], got, _ref(0, 7, off, var, 100003),
                  f"2^64 block carry, phase {ph}")


# variants of two or four words per unit: with the word offset a multiple of
# that, the units lie inside counter blocks and a misaligned output start only
# rotates each block's outputs across two 16-byte groups
MULTIWORD_VARIANTS = [v for v in VARIANTS
                      if v[1] in (2, 3) or (v[2] == 2 and v[1] in (1, 4, 5))]


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("var", MULTIWORD_VARIANTS, ids=[v[0] for v in MULTIWORD_VARIANTS])
def test_misaligned_output_equals_aligned_output(g, engine_kind, var):
    """A fill written at every element offset into a 16-byte group, from word
    offsets that keep the units inside counter blocks (Philox: the rotate
    kernel, lane 0 and lane 31 writing the groups shared by two warps), equals
    the same fill written at an aligned address bit for bit; near the 2^64
    carry of the block counter it equals the oracle."""
    _, kind, dtype, p0, p1 = var
    wpu = 4 if (kind in (2, 3) and dtype == 2) else 2
    es = 8 if dtype == 2 else 4
    n = (1 << 21) + 7
    for off in (0, wpu, 6 * wpu):
        ref = _gpu_fill(g, engine_kind, 2021, off, var, n)
        for pofs in range(1, 16 // es):
            got = _gpu_fill(g, engine_kind, 2021, off, var, n, ptr_off=pofs)
            bad = np.nonzero(_as_uint_view(got) != _as_uint_view(ref))[0]
            assert bad.size == 0, f"{var[0]} off={off} ptr+{pofs}: {bad.size} differ, " \
                                  f"first at {bad[:5]}"
    off = (1 << 66) - 4 * 3000
    for pofs in range(1, 16 // es):
        got = _gpu_fill(g, engine_kind, 11, off, var, 20001, ptr_off=pofs)
        assert_parity(kind, dtype, got, _ref(engine_kind, 11, off, var, 20001),
                      f"{var[0]} 2^64 block carry ptr+{pofs}")


def test_philox_uniform_2pow20_bit_exact(g):
    c = W.PHILOX_UNIFORM_2POW20
    var = c["dist"]
    got = _gpu_fill(g, c["engine"], c["seed"], c["offset"], var, c["n"])
    ref = _ref(c["engine"], c["seed"], c["offset"], var, c["n"])
    assert_parity(var[1], var[2], got, ref, "Philox 2^20 FP32 uniform")


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("var", W.SWEEP_DISTS, ids=[v[0] for v in W.SWEEP_DISTS])
def test_sweep_1e6_full(g, engine_kind, var):
    n = 10**6
    got = _gpu_fill(g, engine_kind, W.SWEEP_SEED, 0, var, n, guard=64)
    ref = _ref(engine_kind, W.SWEEP_SEED, 0, var, n)
    assert_parity(var[1], var[2], got, ref, f"sweep n=1e6 {var[0]}")


def _windows_check(g, engine_kind, var, n, count):
    _, kind, dtype, p0, p1 = var
    out = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
    e = g.Engine(engine_kind, W.SWEEP_SEED, 0)
    g.generate(g.Distribution(kind, dtype, p0, p1), e, out)
    torch.cuda.synchronize()
    assert e.offset == oracle.words_for(kind, dtype, n)
    for start, width in W.sample_windows(n, count=count, width=2048):
        woff = oracle.words_for(kind, dtype, start)
        ref = oracle.generate(engine_kind, W.SWEEP_SEED, woff, kind, dtype, p0, p1, width)
        got = out[start:start + width].cpu().numpy()
        if dtype == 0:
            got = got.view(np.uint32)
        assert_parity(kind, dtype, got, ref, f"{var[0]} n={n} window {start}")
    if kind == 1:  # every uniform lies in [a, b): a property at any size
        assert float(out.min()) >= p0 and float(out.max()) < p1
    del out


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("var", W.SWEEP_DISTS, ids=[v[0] for v in W.SWEEP_DISTS])
def test_sweep_1e7_1e8_windows(g, engine_kind, var):
    for n in (10**7, 10**8):
        _windows_check(g, engine_kind, var, n, count=24)


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("var", W.SWEEP_DISTS, ids=[v[0] for v in W.SWEEP_DISTS])
def test_sweep_1e9_windows(g, engine_kind, var):
    _windows_check(g, engine_kind, var, 10**9, count=24)


@pytest.mark.parametrize("engine_kind,stride", [(1, 1 << 76), (0, 1 << 40)])
def test_16384_substreams(g, engine_kind, stride):
    c = W.SUBSTREAMS
    S, n = c["num_streams"], c["n_per_stream"]
    _, kind, dtype, p0, p1 = c["dist"]
    out = torch.empty(S * n, dtype=torch.float64, device="cuda")
    e = g.Engine(engine_kind, c["seed"], 0)
    g.generate_substreams(g.Distribution(kind, dtype, p0, p1), e, out, n, S, stride)
    torch.cuda.synchronize()
    assert e.offset == 0
    # substreams 0..7 in full: the oracle jumps to s * stride, then steps sequentially
    for s in range(8):
        ref = oracle.generate(engine_kind, c["seed"], s * stride, kind, dtype, p0, p1, n)
        assert_parity(kind, dtype, out[s * n:(s + 1) * n].cpu().numpy(), ref, f"substream {s}")
    # windows in other substreams, including the last
    rng = np.random.Generator(np.random.PCG64(3))
    picks = [S - 1] + [int(x) for x in rng.integers(8, S, size=12)]
    for s in picks:
        start = int(rng.integers(0, n // 2)) * 2
        width = min(512, n - start)
        woff = s * stride + oracle.words_for(kind, dtype, start)
        ref = oracle.generate(engine_kind, c["seed"], woff, kind, dtype, p0, p1, width)
        got = out[s * n + start: s * n + start + width].cpu().numpy()
        assert_parity(kind, dtype, got, ref, f"substream {s} window {start}")


@pytest.mark.parametrize("engine_kind", ENGINES)
def test_substreams_ragged_and_misaligned(g, engine_kind):
    # odd sizes and a misaligned base pointer take the staged / 4-byte-store paths
    for var in [VARIANTS[1], VARIANTS[7], VARIANTS[9], VARIANTS[5]]:
        _, kind, dtype, p0, p1 = var
        S, n, stride = 37, 1001, (1 << 40) + 6
        es = 8 if dtype == 2 else 4
        buf = torch.empty(S * n + 1, dtype=_torch_dtype(dtype), device="cuda")
        out = buf[1:]
        e = g.Engine(engine_kind, 99, 12345)
        g.generate_substreams(g.Distribution(kind, dtype, p0, p1), e, out, n, S, stride)
        torch.cuda.synchronize()
        host = out.cpu().numpy()
        for s in range(S):
            ref = oracle.generate(engine_kind, 99, 12345 + s * stride, kind, dtype, p0, p1, n)
            assert_parity(kind, dtype, host[s * n:(s + 1) * n], ref, f"{var[0]} stream {s}")
        del es


@pytest.mark.parametrize("engine_kind", ENGINES)
def test_continuation_equals_single_call(g, engine_kind):
    """generate(n1); generate(n2) on one engine == generate(n1 + n2) (even n1)."""
    for var in [VARIANTS[0], VARIANTS[2], VARIANTS[4], VARIANTS[7], VARIANTS[9]]:
        _, kind, dtype, p0, p1 = var
        d = g.Distribution(kind, dtype, p0, p1)
        n1, n2 = 1002, 30001
        a = torch.empty(n1 + n2, dtype=_torch_dtype(dtype), device="cuda")
        e = g.Engine(engine_kind, 5, 3)
        g.generate(d, e, a[:n1])
        g.generate(d, e, a[n1:])
        b = torch.empty(n1 + n2, dtype=_torch_dtype(dtype), device="cuda")
        g.generate(d, g.Engine(engine_kind, 5, 3), b)
        torch.cuda.synchronize()
        assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), var[0]
        assert e.offset == 3 + oracle.words_for(kind, dtype, n1 + n2)


@pytest.mark.parametrize("engine_kind", ENGINES)
def test_shards_concatenate_to_unsharded(g, engine_kind):
    """The multi-GPU partition, run shard by shard on one GPU: concatenation of
    the shards is bit-identical to the unsharded fill."""
    from paper_2109_01329_gb300 import shard

    for var in [VARIANTS[1], VARIANTS[7], VARIANTS[9]]:
        _, kind, dtype, p0, p1 = var
        d = g.Distribution(kind, dtype, p0, p1)
        n, world = 1_000_003, 4
        full = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
        g.generate(d, g.Engine(engine_kind, 77, 11), full)
        parts = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
        for r in range(world):
            start, count, woff = shard.shard_range(r, world, n, kind, dtype)
            g.generate(d, g.Engine(engine_kind, 77, 11 + woff), parts[start:start + count])
        torch.cuda.synchronize()
        assert torch.equal(full.view(torch.uint8), parts.view(torch.uint8)), var[0]


def test_generate_host_equals_device(g):
    for engine_kind in ENGINES:
        for var in [VARIANTS[1], VARIANTS[8], VARIANTS[4]]:
            _, kind, dtype, p0, p1 = var
            d = g.Distribution(kind, dtype, p0, p1)
            n = 3_000_001
            dev_out = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
            e1 = g.Engine(engine_kind, 8, 1)
            g.generate(d, e1, dev_out)
            host = torch.empty(n, dtype=_torch_dtype(dtype), pin_memory=True)
            work = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
            e2 = g.Engine(engine_kind, 8, 1)
            g.generate_host(d, e2, host, work)
            assert torch.equal(dev_out.cpu().view(torch.uint8), host.view(torch.uint8)), var[0]
            assert e1.offset == e2.offset


@pytest.mark.parametrize("engine_kind", ENGINES)
def test_seed_word_engines(g, engine_kind):
    """Engines seeded by word lists (including the Philox counter words and
    MRG32k3a full states) against the oracle's independent seeding."""
    rng = np.random.Generator(np.random.PCG64(4))
    for count in range(1, 7):
        words = [int(x) for x in rng.integers(1, 2**32, count)]
        for var in [VARIANTS[0], VARIANTS[1], VARIANTS[7]]:
            _, kind, dtype, p0, p1 = var
            e = g.Engine.from_words(engine_kind, words, offset=3)
            out = torch.empty(1001, dtype=_torch_dtype(dtype), device="cuda")
            g.generate(g.Distribution(kind, dtype, p0, p1), e, out)
            torch.cuda.synchronize()
            ref = oracle.generate_words(engine_kind, words, 3, kind, dtype, p0, p1, 1001)
            got = out.cpu().numpy()
            assert_parity(kind, dtype, got.view(np.uint32) if dtype == 0 else got, ref,
                          f"words {words} {var[0]}")


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("var", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("n,offset,ptr_off", [(3 * (1 << 20) + 5, 0, 0), (1 << 20, 3, 1)])
def test_fill_equals_transform_of_its_words(g, engine_kind, var, n, offset, ptr_off):
    """The fused fill kernels (one counter block per 16-byte group, the staged
    phase, MRG32k3a's chunked copy-out, the inverse CDF's four-at-a-time
    block form) and the transform kernel are separate code; applied to the
    same engine words they must agree bit for bit."""
    _, kind, dtype, p0, p1 = var
    got = _gpu_fill(g, engine_kind, 2021, offset, var, n, ptr_off=ptr_off)
    nw = oracle.words_for(kind, dtype, n)
    words = _gpu_fill(g, engine_kind, 2021, offset, ("bits", 0, 0, 0.0, 0.0), nw)
    w = torch.from_numpy(words.view(np.int32)).cuda()
    out = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
    g.transform_words(g.Distribution(kind, dtype, p0, p1), w, out)
    torch.cuda.synchronize()
    ref = out.cpu().numpy()
    bad = np.nonzero(_as_uint_view(got) != _as_uint_view(ref))[0]
    assert bad.size == 0, f"{var[0]}: {bad.size} differ, first at {bad[:5]}"


def _fill_check(g, e, engine_kind, var, n, ref_fn, what):
    _, kind, dtype, p0, p1 = var
    out = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
    g.generate(g.Distribution(kind, dtype, p0, p1), e, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = ref_fn(kind, dtype, p0, p1, n)
    assert_parity(kind, dtype, got.view(np.uint32) if dtype == 0 else got, ref, what)


@pytest.mark.parametrize("engine_kind", ENGINES)
@pytest.mark.parametrize("seeded_by", ["seed", "words"])
def test_copied_and_restored_engines_continue_the_sequence(g, engine_kind, seeded_by):
    """Copy-constructed engines (oneMKL engines are copy-constructible, Sec. 4.1)
    and engines restored from grng_engine_get_state generate, on the GPU, the
    oracle's outputs from the offset the original had reached; the original
    and its copy are independent afterwards."""
    words = [0x9E3779B9, 17, 0xFFFFFFF0, 5, 6, 0x12345678]
    var_a, var_b = VARIANTS[7], VARIANTS[4]  # gaussian F32, then uniform F64
    if seeded_by == "seed":
        e = g.Engine(engine_kind, 2021, 5)

        def ref_at(off):
            return lambda k, dt, p0, p1, n: oracle.generate(engine_kind, 2021, off, k, dt, p0, p1,
                                                            n)
    else:
        e = g.Engine.from_words(engine_kind, words, offset=5)

        def ref_at(off):
            return lambda k, dt, p0, p1, n: oracle.generate_words(engine_kind, words, off, k, dt,
                                                                  p0, p1, n)
    # move the original mid-stream at an odd word phase; offsets below are
    # relative to the engine's start (a word-seeded Philox engine starts at
    # word 4 * counter + 5)
    start = e.offset
    _fill_check(g, e, engine_kind, var_a, 1001, ref_at(5), "original")
    rel = 5 + 1002
    assert e.offset == start + 1002
    c = e.copy()
    r = g.Engine.restore(e.full_state)
    assert c.full_state == e.full_state == r.full_state
    n = 65537
    for eng, name in ((c, "copy"), (r, "restored"), (e, "original")):
        _fill_check(g, eng, engine_kind, var_b, n, ref_at(rel), name)
    # each advanced by its own call only
    for eng in (c, r, e):
        assert eng.offset == start + 1002 + 2 * n
    _fill_check(g, c, engine_kind, var_a, 777, ref_at(rel + 2 * n), "copy continues")
    assert e.offset == start + 1002 + 2 * n


@pytest.mark.parametrize("engine_kind", ENGINES)
def test_every_fill_geometry_gives_the_same_outputs(g, engine_kind):
    """Every launch geometry the fill autotuner tries gives the same words, bit
    for bit (outputs depend on the word index only); after tuning, fills
    still equal the oracle."""
    cands = [0, 1, 2, 4, 17, 18, 20, 32, 48, 64] if engine_kind == 0 else [0, 1, 2, 4, 6, 12, 16]
    g.tune_reset()
    try:
        for var in [VARIANTS[0], VARIANTS[4], VARIANTS[7], VARIANTS[10], VARIANTS[12]]:
            _, kind, dtype, p0, p1 = var
            d = g.Distribution(kind, dtype, p0, p1)
            n = 1_000_003
            # word offset 5 (the shift kernels), and word offset 4 written one
            # element past a 16-byte boundary (Philox: the rotate kernel for
            # the multi-word variants)
            for off, pofs in ((5, 0), (4, 1)):
                outs = []
                for geo in cands:
                    assert g.fill_geometry(engine_kind, d, n, geo) == geo
                    out = torch.empty(n + pofs, dtype=_torch_dtype(dtype), device="cuda")[pofs:]
                    g.generate(d, g.Engine(engine_kind, 2021, off), out)
                    outs.append(out)
                torch.cuda.synchronize()
                for geo, o in zip(cands[1:], outs[1:]):
                    assert torch.equal(o.view(torch.uint8), outs[0].view(torch.uint8)), \
                        (var[0], off, geo)
            buf = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
            geo, ms, ms0 = g.fill_autotune(engine_kind, d, buf)
            assert geo in cands and 0 < ms <= ms0 * 1.0001
            out = torch.empty(n, dtype=_torch_dtype(dtype), device="cuda")
            g.generate(d, g.Engine(engine_kind, 2021, 5), out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            ref = oracle.generate(engine_kind, 2021, 5, kind, dtype, p0, p1, n)
            assert_parity(kind, dtype, got.view(np.uint32) if dtype == 0 else got, ref, var[0])
    finally:
        g.tune_reset()


@pytest.mark.parametrize("engine_kind,stride", [(1, (1 << 76) + 1), (0, (1 << 40) + 3)])
@pytest.mark.parametrize("var", [VARIANTS[7], VARIANTS[9], VARIANTS[0], VARIANTS[4]],
                         ids=["gauss_f32", "logn_f64", "bits", "u01_f64"])
def test_odd_length_substreams_at_every_phase(g, engine_kind, stride, var):
    """64 substreams of an odd length from a misaligned base, at a word stride
    that is not a multiple of 4: every stream starts at its own 16-byte phase
    and word phase (and, for the Box-Muller fills, every other stream splits a
    pair), over many chunks per stream; streams compared in full with the
    oracle."""
    _, kind, dtype, p0, p1 = var
    S, n = 64, 100_003
    buf = torch.full((S * n + 2,), 0, dtype=_torch_dtype(dtype), device="cuda")
    out = buf[1:1 + S * n]
    e = g.Engine(engine_kind, 77, 9)
    g.generate_substreams(g.Distribution(kind, dtype, p0, p1), e, out, n, S, stride)
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    assert e.offset == 9
    for s in list(range(0, S, 9)) + [S - 1]:
        ref = oracle.generate(engine_kind, 77, 9 + s * stride, kind, dtype, p0, p1, n)
        got = host[s * n:(s + 1) * n]
        assert_parity(kind, dtype, got.view(np.uint32) if dtype == 0 else got, ref,
                      f"{var[0]} stream {s}")
