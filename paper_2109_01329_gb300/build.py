"""Builds libgrng.so in-tree from csrc/ with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  The library exports only the C ABI of
include/grng.h.  Usage: ``python -m paper_2109_01329_gb300.build``.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libgrng.so")
PROBES_PATH = os.path.join(HERE, "libgrng_probes.so")

SOURCES = ["capi.cpp", "philox_kernels.cu", "mrg_kernels.cu", "static_stage.cu",
           "transform_kernels.cu", "batch.cu", "serve.cpp", "tune.cpp"]
HEADERS = ["device_common.cuh", "grng_internal.h", "mrg_tables.h", "bm64_fixed.cuh",
           "bm64_tables.h", "icdf64_fixed.cuh", "icdf64_tables.h", "icdf32_tables.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgrng.so")


def _flags(ptxas_verbose: bool) -> list[str]:
    # host code keeps every multiply and add rounded on its own (no fused
    # forms), as the device code's explicit round-to-nearest intrinsics do
    f = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I", INCLUDE, "-I", CSRC,
         "-Xcompiler", "-fvisibility=hidden"] + ARCH
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def _needs_build() -> bool:
    if not os.path.exists(LIB_PATH) or not os.path.exists(PROBES_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS + ["probes.cu"]]
    deps.append(os.path.join(INCLUDE, "grng.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compiles and links libgrng.so if any source changed; returns its path."""
    if not force and not _needs_build():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    flags = _flags(ptxas_verbose)

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, "-shared"] + ARCH + ["-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    # measurement probes (roofline ceilings for bench.py), a separate library
    pobj = compile_one("probes.cu")
    tmp = PROBES_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([cc, "-shared"] + ARCH + ["-cudart", "static", "-o", tmp, pobj],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"probe link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBES_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
