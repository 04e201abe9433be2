"""CPU oracle for the grng random number path (test infrastructure only).

This package is the plain, slow, sequential reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product library never does.
It shares no code with ``paper_2109_01329_gb300`` and imports nothing from it.

The arithmetic lives in ``grng_oracle.cpp`` (see its header for the readings of
the paper it implements).  This module only builds that file with g++ and
marshals numpy arrays through ctypes.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grng_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
# Test hook: tests/test_oracle_planted.py builds deliberately broken copies of
# the source (one planted mistake each) and runs the pins against them; the
# library of such a copy is built next to it.
if os.environ.get("GRNG_ORACLE_SRC"):
    _SRC = os.path.abspath(os.environ["GRNG_ORACLE_SRC"])
    _LIB = os.path.join(os.path.dirname(_SRC), "liboracle.so")

ENGINE_PHILOX = 0
ENGINE_MRG = 1
DIST_BITS, DIST_UNIFORM, DIST_GAUSSIAN, DIST_LOGNORMAL = 0, 1, 2, 3
DIST_GAUSSIAN_ICDF, DIST_LOGNORMAL_ICDF = 4, 5
DT_U32, DT_F32, DT_F64 = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles grng_oracle.cpp into liboracle.so (no contraction, no SIMD flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_philox4x32_10.restype = None
            L.oracle_words.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int64, u32p]
            L.oracle_words.restype = ctypes.c_int
            L.oracle_mrg_seed_state.argtypes = [ctypes.c_uint64, u64p]
            L.oracle_mrg_seed_state.restype = None
            L.oracle_mrg_step.argtypes = [u64p]
            L.oracle_mrg_step.restype = ctypes.c_uint32
            L.oracle_mrg_skip.argtypes = [u64p, ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_mrg_skip.restype = None
            L.oracle_mrg_matrix_power.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.c_int, u64p]
            L.oracle_mrg_matrix_power.restype = ctypes.c_int
            L.oracle_words_for.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64]
            L.oracle_words_for.restype = ctypes.c_uint64
            L.oracle_u01_f32.argtypes = [ctypes.c_uint32]
            L.oracle_u01_f32.restype = ctypes.c_float
            L.oracle_u01_f64.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_u01_f64.restype = ctypes.c_double
            L.oracle_uniform_f32.argtypes = [ctypes.c_uint32, ctypes.c_float, ctypes.c_float]
            L.oracle_uniform_f32.restype = ctypes.c_float
            L.oracle_uniform_f64.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_double]
            L.oracle_uniform_f64.restype = ctypes.c_double
            L.oracle_transform_words.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int64, u32p,
                                                 ctypes.c_void_p]
            L.oracle_transform_words.restype = ctypes.c_int
            L.oracle_generate.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                          ctypes.c_void_p]
            L.oracle_generate.restype = ctypes.c_int
            L.oracle_generate_words.argtypes = [ctypes.c_int, u32p, ctypes.c_int, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                ctypes.c_void_p]
            L.oracle_generate_words.restype = ctypes.c_int
            _lib = L
    return _lib


def _u32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _split128(v: int):
    v %= 1 << 128
    return v & ((1 << 64) - 1), v >> 64


def philox_block(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def words(engine: int, seed: int, offset: int, n: int) -> np.ndarray:
    """Words [offset, offset + n) of the engine's 32-bit output stream."""
    out = np.empty(max(n, 0), dtype=np.uint32)
    lo, hi = _split128(offset)
    rc = lib().oracle_words(engine, seed & ((1 << 64) - 1), lo, hi, n, _u32p(out))
    if rc != 0:
        raise ValueError("oracle_words: invalid argument")
    return out


def mrg_seed_state(seed: int) -> np.ndarray:
    st = np.empty(6, dtype=np.uint64)
    lib().oracle_mrg_seed_state(seed & ((1 << 64) - 1), _u64p(st))
    return st


def mrg_step(state: np.ndarray) -> int:
    """Steps a six-value MRG32k3a state in place; returns the output word."""
    assert state.dtype == np.uint64 and state.flags.c_contiguous
    return int(lib().oracle_mrg_step(_u64p(state)))


def mrg_skip(state: np.ndarray, k: int) -> None:
    assert state.dtype == np.uint64 and state.flags.c_contiguous
    lo, hi = _split128(k)
    lib().oracle_mrg_skip(_u64p(state), lo, hi)


def mrg_matrix_power(comp: int, e: int) -> np.ndarray:
    """A_comp^e mod m_comp as a 3x3 uint64 matrix (any non-negative exponent)."""
    nbytes = max(1, (e.bit_length() + 7) // 8)
    eb = e.to_bytes(nbytes, "little")
    out = np.empty(9, dtype=np.uint64)
    rc = lib().oracle_mrg_matrix_power(comp, eb, nbytes, _u64p(out))
    if rc != 0:
        raise ValueError("bad component")
    return out.reshape(3, 3)


def words_for(dist: int, dtype: int, n: int) -> int:
    return int(lib().oracle_words_for(dist, dtype, n))


def u01_f32(w: int) -> float:
    return float(lib().oracle_u01_f32(w))


def u01_f64(wa: int, wb: int) -> float:
    return float(lib().oracle_u01_f64(wa, wb))


def uniform_f32(w: int, a: float, b: float) -> np.float32:
    return np.float32(lib().oracle_uniform_f32(w, a, b))


def uniform_f64(wa: int, wb: int, a: float, b: float) -> float:
    return float(lib().oracle_uniform_f64(wa, wb, a, b))


def out_dtype(dist: int, dtype: int):
    """numpy dtype of the oracle's output array for a distribution."""
    if dist == DIST_BITS:
        return np.uint32
    if dist == DIST_UNIFORM:
        return np.float32 if dtype == DT_F32 else np.float64
    return np.float64  # Box-Muller and ICDF families: long double result rounded to double


def transform_words(dist: int, dtype: int, p0: float, p1: float, n: int,
                    w: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.uint32)
    need = words_for(dist, dtype, n)
    if w.size < need:
        raise ValueError(f"need {need} words, got {w.size}")
    out = np.empty(max(n, 0), dtype=out_dtype(dist, dtype))
    rc = lib().oracle_transform_words(dist, dtype, p0, p1, n, _u32p(w), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_transform_words: invalid argument")
    return out


def generate(engine: int, seed: int, offset: int, dist: int, dtype: int, p0: float, p1: float,
             n: int) -> np.ndarray:
    """n outputs of the distribution from the engine at word offset `offset`."""
    out = np.empty(max(n, 0), dtype=out_dtype(dist, dtype))
    lo, hi = _split128(offset)
    rc = lib().oracle_generate(engine, seed & ((1 << 64) - 1), lo, hi, dist, dtype, p0, p1, n,
                               out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_generate: invalid argument")
    return out


def generate_words(engine: int, words, offset: int, dist: int, dtype: int, p0: float, p1: float,
                   n: int) -> np.ndarray:
    """As generate, for an engine seeded by a list of 1..6 32-bit words."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64).astype(np.uint32))
    out = np.empty(max(n, 0), dtype=out_dtype(dist, dtype))
    lo, hi = _split128(offset)
    rc = lib().oracle_generate_words(engine, _u32p(w), int(w.size), lo, hi, dist, dtype, p0, p1,
                                     n, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_generate_words: invalid argument")
    return out
