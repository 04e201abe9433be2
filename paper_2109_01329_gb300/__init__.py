"""grng: bulk random number generation on GB300 (sm_103a).

Engines (Philox4x32-10, MRG32k3a) and distributions (bits, uniform, gaussian
and lognormal by Box-Muller or by the inverse CDF) behind the C ABI of
include/grng.h, implemented by hand-written CUDA kernels in csrc/, with the
batched (Batch) and served (Server) forms.  This package is the thin Python
binding.
"""

from ._binding import (BITS, GAUSSIAN_ICDF, LOGNORMAL_ICDF, Batch, Server, serve_request, F32, F64, GAUSSIAN, LOGNORMAL, MRG32K3A, PHILOX4X32X10, U32,
                       UNIFORM, Distribution, Engine, GrngError, generate, generate_host,
                       generate_host_static,
                       generate_ptr, generate_substreams, load, transform_words, words_for,
                       fill_autotune, fill_geometry, tune_save, tune_load, tune_reset)
from ._binding import LIB_PATH, EXPORTED

__all__ = ["BITS", "GAUSSIAN_ICDF", "LOGNORMAL_ICDF", "Batch", "Server", "serve_request", "F32", "F64", "GAUSSIAN", "LOGNORMAL", "MRG32K3A", "PHILOX4X32X10", "U32",
           "UNIFORM", "Distribution", "Engine", "GrngError", "generate", "generate_host",
           "generate_host_static",
           "generate_ptr", "generate_substreams", "load", "transform_words", "words_for", "LIB_PATH", "EXPORTED",
           "fill_autotune", "fill_geometry", "tune_save", "tune_load", "tune_reset"]
