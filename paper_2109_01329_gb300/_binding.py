"""ctypes binding of libgrng.so (the C ABI of include/grng.h).

Argument marshalling only: every step of generation runs in the library's
CUDA kernels.  PyTorch supplies device memory (tensors) and the current
stream.  There is no CPU fallback: if libgrng.so is missing or cannot be
loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrng.so")

# enums of grng.h
OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUDGET = 1, 2, 3, 4, 5, 6
PHILOX4X32X10 = 0
MRG32K3A = 1
BITS, UNIFORM, GAUSSIAN, LOGNORMAL = 0, 1, 2, 3
GAUSSIAN_ICDF, LOGNORMAL_ICDF = 4, 5
U32, F32, F64 = 0, 1, 2

EXPORTED = ["grng_status_string", "grng_last_error", "grng_engine_create",
            "grng_engine_create_words", "grng_engine_restore",
            "grng_engine_copy", "grng_engine_skip_ahead", "grng_engine_get_state",
            "grng_engine_destroy", "grng_words_for", "grng_generate",
            "grng_generate_substreams", "grng_generate_host", "grng_generate_host_static",
            "grng_transform_words", "grng_batch_workspace_bytes", "grng_batch_create",
            "grng_batch_launch", "grng_batch_autotune", "grng_batch_set_config",
            "grng_batch_commit", "grng_batch_destroy", "grng_server_create",
            "grng_server_submit", "grng_server_wait", "grng_server_release", "grng_server_drain",
            "grng_server_stats", "grng_server_reset_stats", "grng_server_replay",
            "grng_server_destroy", "grng_server_set_release_delay", "grng_fill_autotune",
            "grng_fill_set_geometry", "grng_fill_get_geometry", "grng_tune_save",
            "grng_tune_load", "grng_tune_reset"]


class GrngError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {_status_name(status)}: {detail}")
        self.status = status


class _Dist(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("p0", ctypes.c_double),
                ("p1", ctypes.c_double)]


class _State(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("offset_lo", ctypes.c_uint64),
                ("offset_hi", ctypes.c_uint64), ("words", ctypes.c_uint32 * 6)]


class _Request(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_void_p), ("dist", _Dist), ("n", ctypes.c_int64),
                ("out", ctypes.c_void_p)]


class _ServePart(ctypes.Structure):
    _fields_ = [("dist", _Dist), ("n", ctypes.c_int64)]


class _ServeRequest(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("offset_lo", ctypes.c_uint64),
                ("offset_hi", ctypes.c_uint64), ("num_parts", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("parts", _ServePart * 4)]


class _ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("wall_s", ctypes.c_double),
                ("latency_p50_us", ctypes.c_double), ("latency_p90_us", ctypes.c_double),
                ("latency_p99_us", ctypes.c_double), ("latency_max_us", ctypes.c_double),
                ("latency_mean_us", ctypes.c_double), ("peak_pool_bytes", ctypes.c_double),
                ("mean_batch_requests", ctypes.c_double), ("admit_wait_p50_us", ctypes.c_double),
                ("admit_wait_p99_us", ctypes.c_double), ("admit_wait_max_us", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Loads libgrng.so (built in-tree); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2109_01329_gb300.build` "
                "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.grng_status_string.argtypes = [ctypes.c_int]
        L.grng_status_string.restype = ctypes.c_char_p
        L.grng_last_error.argtypes = []
        L.grng_last_error.restype = ctypes.c_char_p
        L.grng_engine_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.c_uint64]
        L.grng_engine_restore.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_State)]
        L.grng_engine_create_words.argtypes = [ctypes.POINTER(vp), ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32,
                                               ctypes.c_uint64]
        L.grng_engine_copy.argtypes = [ctypes.POINTER(vp), vp]
        L.grng_engine_skip_ahead.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64]
        L.grng_engine_get_state.argtypes = [vp, ctypes.POINTER(_State)]
        L.grng_engine_destroy.argtypes = [vp]
        L.grng_words_for.argtypes = [ctypes.POINTER(_Dist), ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_uint64)]
        L.grng_generate.argtypes = [ctypes.POINTER(_Dist), vp, ctypes.c_int64, vp, vp]
        L.grng_generate_substreams.argtypes = [ctypes.POINTER(_Dist), vp, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                               vp, vp]
        L.grng_generate_host.argtypes = [ctypes.POINTER(_Dist), vp, ctypes.c_int64, vp, vp,
                                         ctypes.c_size_t, vp]
        L.grng_generate_host_static.argtypes = [ctypes.POINTER(_Dist), vp, ctypes.c_int64, vp,
                                                vp]
        L.grng_transform_words.argtypes = [ctypes.POINTER(_Dist), vp, ctypes.c_int64, vp, vp]
        L.grng_batch_workspace_bytes.argtypes = [ctypes.POINTER(_Request), ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        L.grng_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Request),
                                        ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_size_t, vp]
        L.grng_batch_launch.argtypes = [vp, vp]
        L.grng_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_float)]
        L.grng_batch_set_config.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
        L.grng_batch_commit.argtypes = [vp, vp]
        L.grng_batch_destroy.argtypes = [vp]
        L.grng_server_create.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_size_t, ctypes.c_int32,
                                         ctypes.c_int32]
        L.grng_server_submit.argtypes = [vp, ctypes.POINTER(_ServeRequest),
                                         ctypes.POINTER(ctypes.c_uint64)]
        L.grng_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(vp),
                                       ctypes.POINTER(ctypes.c_size_t)]
        L.grng_server_release.argtypes = [vp, ctypes.c_uint64]
        L.grng_server_drain.argtypes = [vp, ctypes.c_int64]
        L.grng_server_stats.argtypes = [vp, ctypes.POINTER(_ServeStats)]
        L.grng_server_reset_stats.argtypes = [vp]
        L.grng_server_replay.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(_ServeRequest), ctypes.c_int64,
                                         ctypes.c_double]
        L.grng_server_destroy.argtypes = [vp]
        L.grng_server_set_release_delay.argtypes = [vp, ctypes.c_int64]
        L.grng_fill_autotune.argtypes = [ctypes.c_int32, ctypes.POINTER(_Dist), ctypes.c_int64, vp,
                                         vp, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_float)]
        L.grng_fill_set_geometry.argtypes = [ctypes.c_int32, ctypes.POINTER(_Dist),
                                             ctypes.c_int64, ctypes.c_int32]
        L.grng_fill_get_geometry.argtypes = [ctypes.c_int32, ctypes.POINTER(_Dist),
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
        L.grng_tune_save.argtypes = [ctypes.c_char_p]
        L.grng_tune_load.argtypes = [ctypes.c_char_p]
        L.grng_tune_reset.argtypes = []
        for name in EXPORTED[2:]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _status_name(status: int) -> str:
    try:
        return load().grng_status_string(status).decode()
    except Exception:  # noqa: BLE001 - naming an error must not raise
        return f"status {status}"


def _check(status: int, where: str) -> None:
    if status != OK:
        detail = load().grng_last_error().decode(errors="replace")
        raise GrngError(status, where, detail)


def _split128(v: int):
    v %= 1 << 128
    return v & ((1 << 64) - 1), v >> 64


@dataclass(frozen=True)
class Distribution:
    """A distribution and its parameters (see grng_distribution in grng.h)."""

    kind: int
    dtype: int
    p0: float = 0.0
    p1: float = 0.0

    def _c(self) -> _Dist:
        return _Dist(self.kind, self.dtype, float(self.p0), float(self.p1))

    @staticmethod
    def bits() -> "Distribution":
        return Distribution(BITS, U32)

    @staticmethod
    def uniform(a: float = 0.0, b: float = 1.0, dtype: int = F32) -> "Distribution":
        return Distribution(UNIFORM, dtype, a, b)

    @staticmethod
    def gaussian(mean: float = 0.0, stddev: float = 1.0, dtype: int = F32) -> "Distribution":
        return Distribution(GAUSSIAN, dtype, mean, stddev)

    @staticmethod
    def lognormal(m: float = 0.0, s: float = 1.0, dtype: int = F32) -> "Distribution":
        return Distribution(LOGNORMAL, dtype, m, s)

    @staticmethod
    def gaussian_icdf(mean: float = 0.0, stddev: float = 1.0, dtype: int = F32) -> "Distribution":
        return Distribution(GAUSSIAN_ICDF, dtype, mean, stddev)

    @staticmethod
    def lognormal_icdf(m: float = 0.0, s: float = 1.0, dtype: int = F32) -> "Distribution":
        return Distribution(LOGNORMAL_ICDF, dtype, m, s)


class Engine:
    """An engine handle (Philox4x32-10 or MRG32k3a) with a 128-bit word offset."""

    def __init__(self, kind: int, seed: int, offset: int = 0, _handle=None):
        L = load()
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            lo, hi = _split128(offset)
            _check(L.grng_engine_create(ctypes.byref(self._h), kind, seed % (1 << 64), lo),
                   "grng_engine_create")
            if hi:
                _check(L.grng_engine_skip_ahead(self._h, 0, hi), "grng_engine_skip_ahead")

    @classmethod
    def from_words(cls, kind: int, words, offset: int = 0) -> "Engine":
        """An engine from a seed initializer list of 1..6 32-bit words."""
        arr = (ctypes.c_uint32 * len(words))(*[int(w) & 0xFFFFFFFF for w in words])
        h = ctypes.c_void_p()
        _check(load().grng_engine_create_words(ctypes.byref(h), kind, arr, len(words),
                                               offset % (1 << 64)), "grng_engine_create_words")
        return cls(kind, 0, _handle=h)

    @property
    def full_state(self) -> dict:
        st = _State()
        _check(load().grng_engine_get_state(self._h, ctypes.byref(st)), "grng_engine_get_state")
        return {"kind": st.kind, "seed": st.seed, "offset": st.offset_lo | (st.offset_hi << 64),
                "words": list(st.words)[: st.reserved]}

    @classmethod
    def restore(cls, state) -> "Engine":
        """From (kind, seed, offset) or a full_state dict."""
        if isinstance(state, dict):
            kind, seed, offset = state["kind"], state["seed"], state["offset"]
            words = state.get("words", [])
        else:
            kind, seed, offset = state
            words = []
        lo, hi = _split128(offset)
        st = _State(kind, len(words), seed % (1 << 64), lo, hi)
        for i, w in enumerate(words):
            st.words[i] = int(w) & 0xFFFFFFFF
        h = ctypes.c_void_p()
        _check(load().grng_engine_restore(ctypes.byref(h), ctypes.byref(st)),
               "grng_engine_restore")
        return cls(kind, 0, _handle=h)

    def copy(self) -> "Engine":
        h = ctypes.c_void_p()
        _check(load().grng_engine_copy(ctypes.byref(h), self._h), "grng_engine_copy")
        return Engine(self.state[0], 0, _handle=h)

    def skip_ahead(self, n: int) -> None:
        lo, hi = _split128(n)
        _check(load().grng_engine_skip_ahead(self._h, lo, hi), "grng_engine_skip_ahead")

    @property
    def state(self) -> tuple:
        st = _State()
        _check(load().grng_engine_get_state(self._h, ctypes.byref(st)), "grng_engine_get_state")
        return (st.kind, st.seed, st.offset_lo | (st.offset_hi << 64))

    @property
    def offset(self) -> int:
        return self.state[2]

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def close(self) -> None:
        if self._h:
            load().grng_engine_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def words_for(dist: Distribution, n: int) -> int:
    out = ctypes.c_uint64()
    d = dist._c()
    _check(load().grng_words_for(ctypes.byref(d), n, ctypes.byref(out)), "grng_words_for")
    return int(out.value)


_TORCH_DTYPES = {}


def _torch_dtype_ok(t, dtype: int) -> bool:
    import torch

    if dtype == F32:
        return t.dtype == torch.float32
    if dtype == F64:
        return t.dtype == torch.float64
    return t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32))


def _stream_ptr(device, stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def generate_ptr(dist: Distribution, engine: Engine, n: int, dev_ptr: int, stream_ptr: int) -> None:
    """grng_generate on a raw device address and a raw cudaStream_t value."""
    d = dist._c()
    _check(load().grng_generate(ctypes.byref(d), engine.handle, n, ctypes.c_void_p(dev_ptr),
                                ctypes.c_void_p(stream_ptr)), "grng_generate")


def generate(dist: Distribution, engine: Engine, out, n: int | None = None, stream=None):
    """Fills a CUDA tensor (contiguous, dtype matching dist) and advances the engine.

    out may be a view at any element offset; n defaults to out.numel().
    Returns out.
    """
    import torch

    if not out.is_cuda:
        raise ValueError("out must be a CUDA tensor")
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    if not _torch_dtype_ok(out, dist.dtype):
        raise ValueError(f"tensor dtype {out.dtype} does not match distribution dtype {dist.dtype}")
    n = out.numel() if n is None else n
    if n > out.numel():
        raise ValueError("n exceeds the tensor size")
    with torch.cuda.device(out.device):
        generate_ptr(dist, engine, n, out.data_ptr(), _stream_ptr(out.device, stream))
    return out


def generate_substreams(dist: Distribution, engine: Engine, out, n_per_stream: int,
                        num_streams: int, stride: int, stream=None):
    """Substream s fills out[s * n_per_stream : (s + 1) * n_per_stream] from word
    offset engine.offset + s * stride.  The engine does not advance."""
    import torch

    if not out.is_cuda or not out.is_contiguous() or not _torch_dtype_ok(out, dist.dtype):
        raise ValueError("out must be a contiguous CUDA tensor of the distribution's dtype")
    if n_per_stream * num_streams > out.numel():
        raise ValueError("out is too small")
    lo, hi = _split128(stride)
    d = dist._c()
    with torch.cuda.device(out.device):
        _check(load().grng_generate_substreams(ctypes.byref(d), engine.handle, n_per_stream,
                                               num_streams, lo, hi,
                                               ctypes.c_void_p(out.data_ptr()),
                                               ctypes.c_void_p(_stream_ptr(out.device, stream))),
               "grng_generate_substreams")
    return out


def generate_host(dist: Distribution, engine: Engine, host_out, work, stream=None,
                  n: int | None = None):
    """grng_generate_host: fills a CPU tensor through the device buffer `work`
    (a CUDA tensor of at least 2 MiB).  Synchronous."""
    import torch

    if host_out.is_cuda or not host_out.is_contiguous() or not _torch_dtype_ok(host_out,
                                                                                 dist.dtype):
        raise ValueError("host_out must be a contiguous CPU tensor of the distribution's dtype")
    n = host_out.numel() if n is None else n
    if n < 0 or n > host_out.numel():
        raise ValueError(f"n = {n} outside [0, host_out.numel() = {host_out.numel()}]")
    if not work.is_cuda:
        raise ValueError("work must be a CUDA tensor")
    d = dist._c()
    nbytes = work.numel() * work.element_size()
    with torch.cuda.device(work.device):
        _check(load().grng_generate_host(ctypes.byref(d), engine.handle, n,
                                         ctypes.c_void_p(host_out.data_ptr()),
                                         ctypes.c_void_p(work.data_ptr()), nbytes,
                                         ctypes.c_void_p(_stream_ptr(work.device, stream))),
               "grng_generate_host")
    return host_out


def _header_stage_bytes() -> int:
    """GRNG_STATIC_STAGE_BYTES as include/grng.h defines it (one source of truth)."""
    import re

    path = os.path.join(os.path.dirname(HERE), "include", "grng.h")
    with open(path) as f:
        m = re.search(r"#define\s+GRNG_STATIC_STAGE_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", f.read())
    if m is None:
        raise RuntimeError("GRNG_STATIC_STAGE_BYTES not found in include/grng.h")
    return int(m.group(1)) << int(m.group(2))


STATIC_STAGE_BYTES = _header_stage_bytes()


def generate_host_static(dist: Distribution, engine: Engine, host_out, n: int | None = None,
                         stream=None, device=None):
    """grng_generate_host_static: fills a CPU tensor through the library's own
    static device staging array (no allocation; n * element size must not
    exceed STATIC_STAGE_BYTES).  Synchronous."""
    import torch

    if host_out.is_cuda or not host_out.is_contiguous() or not _torch_dtype_ok(host_out,
                                                                                 dist.dtype):
        raise ValueError("host_out must be a contiguous CPU tensor of the distribution's dtype")
    n = host_out.numel() if n is None else n
    if n < 0 or n > host_out.numel():
        raise ValueError(f"n = {n} outside [0, host_out.numel() = {host_out.numel()}]")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    d = dist._c()
    with torch.cuda.device(dev):
        _check(load().grng_generate_host_static(ctypes.byref(d), engine.handle, n,
                                                ctypes.c_void_p(host_out.data_ptr()),
                                                ctypes.c_void_p(_stream_ptr(dev, stream))),
               "grng_generate_host_static")
    return host_out


def fill_autotune(engine_kind: int, dist: Distribution, buf, n: int | None = None,
                  stream=None):
    """grng_fill_autotune: times the candidate launch geometries of a fill of n
    outputs into the CUDA tensor buf and keeps the fastest for n's size
    bucket; returns (geometry, ms, ms of the built-in geometry)."""
    import torch

    if not buf.is_cuda or not _torch_dtype_ok(buf, dist.dtype):
        raise ValueError("buf must be a CUDA tensor of the distribution's dtype")
    n = buf.numel() if n is None else n
    if n < 1 or n > buf.numel():
        raise ValueError("n outside [1, buf.numel()]")
    d = dist._c()
    geo, ms, ms0 = ctypes.c_int32(), ctypes.c_float(), ctypes.c_float()
    with torch.cuda.device(buf.device):
        _check(load().grng_fill_autotune(engine_kind, ctypes.byref(d), n,
                                         ctypes.c_void_p(buf.data_ptr()),
                                         ctypes.c_void_p(_stream_ptr(buf.device, stream)),
                                         ctypes.byref(geo), ctypes.byref(ms), ctypes.byref(ms0)),
               "grng_fill_autotune")
    return geo.value, ms.value, ms0.value


def fill_geometry(engine_kind: int, dist: Distribution, n: int, geometry: int | None = None) -> int:
    """Reads (or, with geometry, sets) the launch geometry of n's size bucket."""
    d = dist._c()
    if geometry is not None:
        _check(load().grng_fill_set_geometry(engine_kind, ctypes.byref(d), n, geometry),
               "grng_fill_set_geometry")
    g = ctypes.c_int32()
    _check(load().grng_fill_get_geometry(engine_kind, ctypes.byref(d), n, ctypes.byref(g)),
           "grng_fill_get_geometry")
    return g.value


def tune_save(path: str) -> None:
    _check(load().grng_tune_save(os.fsencode(path)), "grng_tune_save")


def tune_load(path: str) -> None:
    _check(load().grng_tune_load(os.fsencode(path)), "grng_tune_load")


def tune_reset() -> None:
    _check(load().grng_tune_reset(), "grng_tune_reset")


def transform_words(dist: Distribution, words, out, n: int | None = None, stream=None):
    """grng_transform_words: applies dist to the device words tensor (int32 / uint32)."""
    import torch

    if not (words.is_cuda and out.is_cuda and words.is_contiguous() and out.is_contiguous()):
        raise ValueError("words and out must be contiguous CUDA tensors")
    if not _torch_dtype_ok(out, dist.dtype):
        raise ValueError("out dtype does not match the distribution")
    n = out.numel() if n is None else n
    if words.numel() * words.element_size() < 4 * words_for(dist, n):
        raise ValueError("not enough words")
    d = dist._c()
    with torch.cuda.device(out.device):
        _check(load().grng_transform_words(ctypes.byref(d), ctypes.c_void_p(words.data_ptr()), n,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(_stream_ptr(out.device, stream))),
               "grng_transform_words")
    return out


class Batch:
    """A planned batch of requests (grng_batch_*).

    requests: list of (engine, distribution, out_tensor[, n]).  The device
    workspace is allocated here as a torch tensor and kept alive with the
    batch; with tunable=True it is sized for ipt = 1, so that autotune() may
    try every geometry.  launch() enqueues the persistent fill and the
    device-side offset advance (capturable in a CUDA graph); commit() moves
    the engines to the device-resident offsets.
    """

    def __init__(self, requests, ipt: int = 8, stream=None, tunable: bool = True):
        import torch

        self._reqs = list(requests)
        arr = (_Request * len(self._reqs))()
        self._keep = []
        dev = None
        for i, r in enumerate(self._reqs):
            engine, dist, out = r[0], r[1], r[2]
            n = r[3] if len(r) > 3 else out.numel()
            if not out.is_cuda or not _torch_dtype_ok(out, dist.dtype):
                raise ValueError(f"request {i}: out must be a CUDA tensor of the dtype")
            dev = out.device
            arr[i].engine = engine.handle
            arr[i].dist = dist._c()
            arr[i].n = n
            arr[i].out = out.data_ptr()
            self._keep.append((engine, out))
        self._arr = arr
        L = load()
        nbytes = ctypes.c_size_t()
        _check(L.grng_batch_workspace_bytes(arr, len(arr), 1 if tunable else ipt,
                                            ctypes.byref(nbytes)), "grng_batch_workspace_bytes")
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
        self._dev = dev
        self._h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(L.grng_batch_create(ctypes.byref(self._h), arr, len(arr), ipt,
                                       ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                       ctypes.c_void_p(_stream_ptr(dev, stream))),
                   "grng_batch_create")

    def launch(self, stream=None):
        import torch

        with torch.cuda.device(self._dev):
            _check(load().grng_batch_launch(self._h, ctypes.c_void_p(_stream_ptr(self._dev, stream))),
                   "grng_batch_launch")

    def autotune(self, stream=None):
        """(ipt, CTAs per SM, ms per fill) of the fastest geometry, now in use."""
        import torch

        i, c, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        with torch.cuda.device(self._dev):
            _check(load().grng_batch_autotune(self._h, ctypes.c_void_p(_stream_ptr(self._dev, stream)),
                                              ctypes.byref(i), ctypes.byref(c), ctypes.byref(ms)),
                   "grng_batch_autotune")
        return i.value, c.value, ms.value

    def set_config(self, ipt: int, ctas_per_sm: int, stream=None):
        import torch

        with torch.cuda.device(self._dev):
            _check(load().grng_batch_set_config(self._h, ipt, ctas_per_sm,
                                                ctypes.c_void_p(_stream_ptr(self._dev, stream))),
                   "grng_batch_set_config")

    def commit(self, stream=None):
        import torch

        with torch.cuda.device(self._dev):
            _check(load().grng_batch_commit(self._h, ctypes.c_void_p(_stream_ptr(self._dev, stream))),
                   "grng_batch_commit")

    def close(self):
        if self._h:
            load().grng_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


SERVE_AUTO_RELEASE = 1


def serve_request(seed: int, parts, offset: int = 0) -> _ServeRequest:
    """A server request: parts = [(Distribution, n), ...] (1..4) from one Philox engine."""
    if not 1 <= len(parts) <= 4:
        raise ValueError("1 to 4 parts")
    q = _ServeRequest()
    q.seed = seed % (1 << 64)
    q.offset_lo, q.offset_hi = _split128(offset)
    q.num_parts = len(parts)
    for k, (d, n) in enumerate(parts):
        q.parts[k].dist = d._c()
        q.parts[k].n = n
    return q


class Server:
    """Continuous-batching server (grng_server_*) over a device pool tensor."""

    def __init__(self, pool_bytes: int, num_streams: int = 2, auto_release: bool = False,
                 device=None):
        import torch

        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(load().grng_server_create(ctypes.byref(self._h),
                                             ctypes.c_void_p(self.pool.data_ptr()), pool_bytes,
                                             num_streams, SERVE_AUTO_RELEASE if auto_release else 0),
                   "grng_server_create")

    def submit(self, req: _ServeRequest) -> int:
        t = ctypes.c_uint64()
        _check(load().grng_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)),
               "grng_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_s: float = 30.0):
        """(device address, bytes) of a completed request's output."""
        p, b = ctypes.c_void_p(), ctypes.c_size_t()
        _check(load().grng_server_wait(self._h, ticket, int(timeout_s * 1e6), ctypes.byref(p),
                                       ctypes.byref(b)), "grng_server_wait")
        return p.value, b.value

    def output(self, ticket: int, timeout_s: float = 30.0):
        """The completed request's output bytes as a view of the pool tensor."""
        addr, nbytes = self.wait(ticket, timeout_s)
        off = addr - self.pool.data_ptr()
        return self.pool[off:off + nbytes]

    def release(self, ticket: int) -> None:
        _check(load().grng_server_release(self._h, ticket), "grng_server_release")

    def drain(self, timeout_s: float = 120.0) -> None:
        _check(load().grng_server_drain(self._h, int(timeout_s * 1e6)), "grng_server_drain")

    def stats(self) -> dict:
        s = _ServeStats()
        _check(load().grng_server_stats(self._h, ctypes.byref(s)), "grng_server_stats")
        return {k: getattr(s, k) for k, _ in _ServeStats._fields_}

    def reset_stats(self) -> None:
        _check(load().grng_server_reset_stats(self._h), "grng_server_reset_stats")

    def set_release_delay(self, seconds: float) -> None:
        """With auto_release: each output stays in the budget this long after
        completion (a consumer holding it), so the budget can bind."""
        _check(load().grng_server_set_release_delay(self._h, int(seconds * 1e6)),
               "grng_server_set_release_delay")

    def replay(self, arrivals, requests, time_scale: float = 1.0) -> None:
        n = len(requests)
        arr = (ctypes.c_double * n)(*[float(a) for a in arrivals])
        rq = (_ServeRequest * n)(*requests)
        _check(load().grng_server_replay(self._h, arr, rq, n, time_scale), "grng_server_replay")

    def close(self) -> None:
        if self._h:
            load().grng_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
