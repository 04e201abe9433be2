"""The C ABI without a GPU: the library loads, exports every function that
include/grng.h declares, and its host-side logic (engines, offsets, the
consumption rule, argument checks) behaves as documented.  No call here
reaches a kernel launch."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    import __graft_entry__  # noqa: F401  (build helper lives there)
    from paper_2109_01329_gb300 import build

    build.build()
    import paper_2109_01329_gb300 as grng

    grng.load()
    return grng


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "grng.h")).read()
    return sorted(set(re.findall(r"GRNG_API\s+[\w\s\*]+?\b(grng_\w+)\s*\(", src)))


def test_header_declares_expected_functions():
    decl = _declared_functions()
    assert "grng_generate" in decl and "grng_engine_create" in decl
    assert len(decl) >= 12


def test_library_exports_every_declared_function(g):
    lib = g.load()
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert sorted(g.EXPORTED) == sorted(_declared_functions())


def test_status_strings(g):
    lib = g.load()
    assert lib.grng_status_string(0) == b"GRNG_OK"
    assert lib.grng_status_string(4) == b"GRNG_ERR_CUDA"
    assert lib.grng_status_string(99) == b"GRNG_ERR_UNKNOWN"


@pytest.mark.parametrize("dist,n", [((0, 0), 7), ((1, 1), 5), ((1, 2), 5), ((2, 1), 5),
                                    ((2, 2), 5), ((3, 1), 1), ((3, 2), 2), ((2, 1), 0)])
def test_words_for_matches_oracle(g, dist, n):
    kind, dtype = dist
    d = g.Distribution(kind, dtype, 0.0, 1.0)
    assert g.words_for(d, n) == oracle.words_for(kind, dtype, n)


def test_engine_state_offsets_and_skip(g):
    e = g.Engine(g.PHILOX4X32X10, 2021, 17)
    assert e.state == (g.PHILOX4X32X10, 2021, 17)
    e.skip_ahead(2**76 + 3)
    assert e.offset == 17 + 2**76 + 3
    e.skip_ahead(2**128 - 1)  # wraps mod 2^128
    assert e.offset == 17 + 2**76 + 2
    c = e.copy()
    c.skip_ahead(1)
    assert c.offset == e.offset + 1
    r = g.Engine.restore((g.MRG32K3A, 5, 2**100))
    assert r.state == (g.MRG32K3A, 5, 2**100)


def test_zero_size_is_noop_and_keeps_offset(g):
    e = g.Engine(g.MRG32K3A, 1, 8)
    g.generate_ptr(g.Distribution.uniform(), e, 0, 0, 0)
    assert e.offset == 8


@pytest.mark.parametrize("dist", [
    (0, 1, 0.0, 1.0),      # bits with F32
    (1, 0, 0.0, 1.0),      # uniform with U32
    (1, 1, 1.0, 1.0),      # a == b
    (1, 1, 2.0, 1.0),      # a > b
    (1, 1, -3.5e38, 3.5e38),  # b - a overflows float
    (1, 2, float("nan"), 1.0),
    (2, 1, 0.0, 0.0),      # stddev 0
    (2, 2, 0.0, -1.0),
    (3, 1, 0.0, float("inf")),
    (7, 1, 0.0, 1.0),      # unknown kind
])
def test_invalid_distributions_rejected_engine_unchanged(g, dist):
    e = g.Engine(g.PHILOX4X32X10, 3, 0)
    with pytest.raises(g.GrngError) as ei:
        g.generate_ptr(g.Distribution(*dist), e, 16, 0x100000, 0)
    assert ei.value.status == 1
    assert e.offset == 0


def test_invalid_pointer_and_size(g):
    e = g.Engine(g.PHILOX4X32X10, 3, 0)
    with pytest.raises(g.GrngError):  # NULL with n > 0
        g.generate_ptr(g.Distribution.uniform(), e, 4, 0, 0)
    with pytest.raises(g.GrngError):  # F32 pointer not 4-byte aligned
        g.generate_ptr(g.Distribution.uniform(), e, 4, 0x100002, 0)
    with pytest.raises(g.GrngError):  # F64 pointer not 8-byte aligned
        g.generate_ptr(g.Distribution.uniform(dtype=g.F64), e, 4, 0x100004, 0)
    with pytest.raises(g.GrngError):
        g.generate_ptr(g.Distribution.uniform(), e, -1, 0x100000, 0)
    with pytest.raises(g.GrngError) as ei:
        g.generate_ptr(g.Distribution.uniform(), e, (1 << 40) + 1, 0x100000, 0)
    assert ei.value.status == 2
    assert e.offset == 0


def test_null_engine_and_create_errors(g):
    lib = g.load()
    d = g.Distribution.uniform()._c()
    assert lib.grng_generate(ctypes.byref(d), None, 4, ctypes.c_void_p(0x1000), None) == 1
    h = ctypes.c_void_p()
    assert lib.grng_engine_create(ctypes.byref(h), 9, 1, 0) == 1
    assert lib.grng_engine_create(None, 0, 1, 0) == 1
    assert lib.grng_engine_destroy(None) == 0
    assert lib.grng_words_for(None, 4, None) == 1


def test_substream_limits(g):
    lib = g.load()
    e = g.Engine(g.MRG32K3A, 1, 0)
    d = g.Distribution.gaussian(dtype=g.F64)._c()
    st = lib.grng_generate_substreams(ctypes.byref(d), e.handle, 1 << 30, 1 << 20, 0, 1 << 12,
                                      ctypes.c_void_p(0x1000), None)
    assert st == 2
    st = lib.grng_generate_substreams(ctypes.byref(d), e.handle, 0, 5, 0, 1,
                                      ctypes.c_void_p(0), None)
    assert st == 0
    assert e.offset == 0


def test_server_argument_errors(g):
    lib = g.load()
    h = ctypes.c_void_p()
    # NULL pool, misaligned pool, bad stream counts: refused before any CUDA call
    assert lib.grng_server_create(ctypes.byref(h), None, 1 << 30, 2, 0) == 1
    assert lib.grng_server_create(ctypes.byref(h), ctypes.c_void_p(0x1001), 1 << 30, 2, 0) == 1
    assert lib.grng_server_create(ctypes.byref(h), ctypes.c_void_p(0x1000), 1 << 30, 0, 0) == 1
    assert lib.grng_server_create(ctypes.byref(h), ctypes.c_void_p(0x1000), 1 << 30, 9, 0) == 1
    assert lib.grng_server_create(ctypes.byref(h), ctypes.c_void_p(0x1000), 1 << 10, 2, 0) == 1
    assert lib.grng_server_destroy(None) == 0
    t = ctypes.c_uint64()
    assert lib.grng_server_submit(None, None, ctypes.byref(t)) == 1


def test_batch_argument_errors(g):
    lib = g.load()
    nbytes = ctypes.c_size_t()
    assert lib.grng_batch_workspace_bytes(None, 1, 4, ctypes.byref(nbytes)) == 1
    e = g.Engine(g.MRG32K3A, 1, 0)
    req = (g._binding._Request * 1)()
    req[0].engine = e.handle
    req[0].dist = g.Distribution.uniform()._c()
    req[0].n = 16
    req[0].out = 0x100000
    assert lib.grng_batch_workspace_bytes(req, 1, 4, ctypes.byref(nbytes)) == 2  # MRG: unsupported
    pe = g.Engine(g.PHILOX4X32X10, 1, 0)
    req[0].engine = pe.handle
    assert lib.grng_batch_workspace_bytes(req, 1, 4, ctypes.byref(nbytes)) == 0
    assert nbytes.value >= 256
    assert lib.grng_batch_workspace_bytes(req, 1, 0, ctypes.byref(nbytes)) == 1  # ipt out of range
    assert lib.grng_batch_destroy(None) == 0


def test_seed_words_engines(g):
    e = g.Engine.from_words(g.MRG32K3A, [5, 6, 7, 8], offset=100)
    st = e.full_state
    assert st["words"] == [5, 6, 7, 8] and st["offset"] == 100
    r = g.Engine.restore(st)
    assert r.full_state == st
    p = g.Engine.from_words(g.PHILOX4X32X10, [1, 2, 3], offset=5)
    assert p.state == (g.PHILOX4X32X10, 1 | (2 << 32), 4 * 3 + 5)
    lib = g.load()
    h = ctypes.c_void_p()
    zeros = (ctypes.c_uint32 * 6)(0, 0, 0, 1, 1, 1)
    assert lib.grng_engine_create_words(ctypes.byref(h), g.MRG32K3A, zeros, 6, 0) == 1
    assert lib.grng_engine_create_words(ctypes.byref(h), g.MRG32K3A, zeros, 0, 0) == 1
    assert lib.grng_engine_create_words(ctypes.byref(h), g.MRG32K3A, zeros, 7, 0) == 1
    m = (ctypes.c_uint32 * 1)(4294967087)  # m1 = 0 mod m1
    assert lib.grng_engine_create_words(ctypes.byref(h), g.MRG32K3A, m, 1, 0) == 0  # (1, 1, 0) is fine


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("words", [1, 6, 2**33 + 5, 2**70 + 3])
def test_skip_back_by_wrapping_restores_the_state(g, kind, words):
    """Moving an engine back by w words as a skip of 2^128 - w (the rollback of
    grng_generate_host_static after a failed copy) restores its state exactly,
    for word-seeded MRG32k3a engines too."""
    engines = [g.Engine(kind, 2021, 11)]
    if kind == 1:
        engines.append(g.Engine.from_words(kind, [5, 6, 7, 8, 9, 10], 11))
    for e in engines:
        before = e.full_state
        e.skip_ahead(words)
        assert e.offset == (11 + words) % (1 << 128)
        back = (1 << 128) - words  # below 2^64 words this is the rollback's (~w + 1, ~0)
        lo, hi = back & ((1 << 64) - 1), back >> 64
        lib = g.load()
        assert lib.grng_engine_skip_ahead(e.handle, lo, hi) == 0
        assert e.full_state == before


def test_host_wrappers_refuse_n_beyond_the_tensor(g):
    """n larger than the host tensor is refused before any copy is made."""
    import torch

    d = g.Distribution.uniform(0.0, 1.0, g.F32)
    e = g.Engine(0, 1, 0)
    host = torch.empty(4, dtype=torch.float32)
    with pytest.raises(ValueError):
        g.generate_host(d, e, host, work=host, n=5)
    with pytest.raises(ValueError):
        g.generate_host_static(d, e, host, n=5)
    with pytest.raises(ValueError):
        g.generate_host_static(d, e, host, n=-1)
    assert e.offset == 0


def test_tune_table_save_load_reset(g, tmp_path):
    """The launch-geometry table: set, save, reset, load back; bad files and
    bad arguments are refused (no GPU work involved)."""
    d32 = g.Distribution.uniform(0.0, 1.0, g.F32)
    d64 = g.Distribution.gaussian(0.0, 1.0, g.F64)
    g.tune_reset()
    assert g.fill_geometry(0, d32, 10**9) == 0
    assert g.fill_geometry(0, d32, 10**9, 4) == 4
    assert g.fill_geometry(1, d64, 1000, 12) == 12
    # same bucket (bit length) shares the entry; another bucket does not
    assert g.fill_geometry(0, d32, 2**29 + 1) == 4
    assert g.fill_geometry(0, d32, 2**31) == 0
    path = str(tmp_path / "tune.txt")
    g.tune_save(path)
    text = open(path).read().split("\n")
    assert text[0] == "grng-tune 1" and len([x for x in text[1:] if x]) == 2
    g.tune_reset()
    assert g.fill_geometry(0, d32, 10**9) == 0
    g.tune_load(path)
    assert g.fill_geometry(0, d32, 10**9) == 4 and g.fill_geometry(1, d64, 1000) == 12
    bad = tmp_path / "bad.txt"
    bad.write_text("grng-tune 1\n0 99 3 4\n")
    with pytest.raises(g.GrngError):
        g.tune_load(str(bad))
    bad.write_text("something else\n")
    with pytest.raises(g.GrngError):
        g.tune_load(str(bad))
    with pytest.raises(g.GrngError):
        g.fill_geometry(0, d32, 100, 65)
    with pytest.raises(g.GrngError):
        g.fill_geometry(2, d32, 100, 1)
    g.tune_reset()


def test_tune_cache_from_the_environment(g, tmp_path):
    """A cache file named by GRNG_TUNE_CACHE is read when the table is first
    used (in a fresh process); a missing file is no error."""
    import subprocess
    import sys

    path = tmp_path / "cache.txt"
    d = g.Distribution.uniform(0.0, 1.0, g.F32)
    g.tune_reset()
    g.fill_geometry(1, d, 5000, 6)
    g.tune_save(str(path))
    g.tune_reset()
    code = ("import paper_2109_01329_gb300 as g; "
            "d = g.Distribution.uniform(0.0, 1.0, g.F32); "
            "print(g.fill_geometry(1, d, 5000), g.fill_geometry(0, d, 5000))")
    env = dict(os.environ, GRNG_TUNE_CACHE=str(path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=120, check=True).stdout.split()
    assert out == ["6", "0"]
    env["GRNG_TUNE_CACHE"] = str(tmp_path / "missing.txt")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=120, check=True).stdout.split()
    assert out == ["0", "0"]
