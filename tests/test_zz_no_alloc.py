"""grng_generate_host_static: generate-to-host with no allocation.

Some callers cannot allocate device memory when they need random numbers (a
host application whose memory pool already owns the device, code that must
not risk the device synchronisation cudaMalloc / cudaFree can cause, plug-ins
whose host forbids device allocations after start-up).  For them the library
stages through its own fixed device array.  This file checks, through the C
ABI, that two calls in a row give the same values as the allocating path
(grng_generate into a device tensor, then a copy), that the engine advances
identically, and that requests above the array's size are refused with the
engine untouched.  It is collected last so that a failure here does not hide
any other test.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# GRNG_STATIC_STAGE_BYTES, read from include/grng.h by the binding
from paper_2109_01329_gb300._binding import STATIC_STAGE_BYTES as STAGE_BYTES  # noqa: E402


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2109_01329_gb300 as grng

    return grng


def _static_call(g, dist, engine, host):
    lib = g.load()
    d = dist._c()
    stream = torch.cuda.current_stream().cuda_stream
    return lib.grng_generate_host_static(ctypes.byref(d), engine.handle, host.numel(),
                                         ctypes.c_void_p(host.data_ptr()),
                                         ctypes.c_void_p(stream))


def _close(kind, dtype, a: np.ndarray, b: np.ndarray) -> bool:
    if kind in (0, 1):  # bits and uniform: bit-exact
        return np.array_equal(a.view(np.uint8), b.view(np.uint8))
    tol = 2e-6 if dtype == 1 else 1e-14
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    return bool(np.all(np.abs(a64 - b64) <= tol * np.maximum(1.0, np.abs(b64))))


CASES = [(0, 0, 0.0, 0.0, 1_000_003), (1, 1, 0.0, 1.0, 4_194_301), (2, 1, 0.0, 1.0, 999_999),
         (1, 2, -1.0, 1.0, 2_000_001), (2, 2, 0.0, 1.0, 65_537), (3, 1, 0.0, 1.0, 5)]


@pytest.mark.parametrize("engine_kind", [0, 1])
def test_static_matches_allocating_path_two_calls(g, engine_kind):
    tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}
    for kind, dtype, p0, p1, n in CASES:
        dist = g.Distribution(kind, dtype, p0, p1)
        e_static = g.Engine(engine_kind, 2021, 7)
        e_ref = g.Engine(engine_kind, 2021, 7)
        for call in range(2):  # two calls in a row continue the same sequence
            host = torch.empty(n, dtype=tdt[dtype])
            assert _static_call(g, dist, e_static, host) == 0, g.load().grng_last_error()
            dev = torch.empty(n, dtype=tdt[dtype], device="cuda")
            g.generate(dist, e_ref, dev)
            ref = dev.cpu().numpy()
            assert _close(kind, dtype, host.numpy(), ref), (kind, dtype, call)
            assert e_static.offset == e_ref.offset


def test_size_limit_refused_engine_unchanged(g):
    e = g.Engine(0, 1, 0)
    too_big = STAGE_BYTES // 8 + 1
    host = torch.empty(too_big, dtype=torch.float64)
    st = _static_call(g, g.Distribution(1, 2, 0.0, 1.0), e, host)
    assert st == 2  # GRNG_ERR_UNSUPPORTED
    assert b"static staging" in g.load().grng_last_error()
    assert e.offset == 0
    # exactly at the limit is accepted
    host = torch.empty(STAGE_BYTES // 4, dtype=torch.float32)
    assert _static_call(g, g.Distribution(1, 1, 0.0, 1.0), e, host) == 0
    assert e.offset == STAGE_BYTES // 4


def test_python_wrapper_two_calls(g):
    """The binding's generate_host_static: two calls continue one sequence and
    equal grng_generate; an n beyond the host tensor is refused before any
    copy could write past it."""
    d = g.Distribution.uniform(0.0, 1.0, g.F32)
    e_static, e_ref = g.Engine(1, 99, 3), g.Engine(1, 99, 3)
    for _ in range(2):
        host = torch.empty(10_001, dtype=torch.float32)
        g.generate_host_static(d, e_static, host)
        dev = torch.empty(10_001, dtype=torch.float32, device="cuda")
        g.generate(d, e_ref, dev)
        assert np.array_equal(host.numpy().view(np.uint32), dev.cpu().numpy().view(np.uint32))
    with pytest.raises(ValueError):
        g.generate_host_static(d, e_static, torch.empty(4, dtype=torch.float32), n=5)
    assert e_static.offset == e_ref.offset
