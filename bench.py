"""Benchmark: the single-stream fill sweep at n = 10^9.

One step = one pass of the whole path over the sweep workload: for each engine
(Philox4x32-10, MRG32k3a) and each distribution (bits U32, uniform F32 and F64
on [0, 1), Box-Muller gaussian F32 and F64, lognormal F32), create an engine
(seed 2021, offset = this rank's shard), generate n outputs into a resident
device buffer (the output of every fill, 4 or 8 GB, is far larger than L2) and
advance the engine.  value = samples of all ranks / step time (Gsamples/s).

Beside it: per-kernel achieved HBM write GB/s against the measured copy peak,
the roofline of the dominant kernel, cuRAND's host API on the same fills
(the native baseline of the paper, Sec. 4.2), an end-to-end number through
the C ABI with host buffers (generate + device-to-host copy), clocks sampled
during the timed region, and the CPU oracle as the timed CPU baseline.

--impl reference times the oracle (plain CPU C++) on the host cores instead.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2109_01329_gb300 import workloads as W  # noqa: E402

METRIC = "Gsamples/s and HBM-write GB/s (fraction of roofline) vs cuRAND; batched p50/p99"
UNIT = "Gsamples/s"
ENGINES = [(0, "philox4x32_10"), (1, "mrg32k3a")]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- cuRAND
class Curand:
    """cuRAND host API through ctypes: the native baseline (timing only)."""

    RNG = {0: 161, 1: 121}  # CURAND_RNG_PSEUDO_PHILOX4_32_10, CURAND_RNG_PSEUDO_MRG32K3A

    def __init__(self):
        lib = None
        for name in ("libcurand.so", "libcurand.so.10"):
            for d in ("", "/usr/local/cuda/lib64/", "/usr/local/cuda/targets/sbsa-linux/lib/"):
                try:
                    lib = ctypes.CDLL(d + name)
                    break
                except OSError:
                    continue
            if lib:
                break
        if lib is None:
            raise RuntimeError("libcurand not found")
        self.lib = lib
        vp = ctypes.c_void_p
        lib.curandCreateGenerator.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
        lib.curandSetPseudoRandomGeneratorSeed.argtypes = [vp, ctypes.c_ulonglong]
        lib.curandSetStream.argtypes = [vp, vp]
        lib.curandDestroyGenerator.argtypes = [vp]
        lib.curandGenerate.argtypes = [vp, vp, ctypes.c_size_t]
        lib.curandGenerateUniform.argtypes = [vp, vp, ctypes.c_size_t]
        lib.curandGenerateUniformDouble.argtypes = [vp, vp, ctypes.c_size_t]
        lib.curandGenerateNormal.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_float,
                                             ctypes.c_float]
        lib.curandGenerateNormalDouble.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_double,
                                                   ctypes.c_double]
        lib.curandGenerateLogNormal.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_float,
                                                ctypes.c_float]

    def generator(self, engine: int, seed: int, stream_ptr: int):
        g = ctypes.c_void_p()
        st = self.lib.curandCreateGenerator(ctypes.byref(g), self.RNG[engine])
        if st != 0:
            raise RuntimeError(f"curandCreateGenerator: {st}")
        self.lib.curandSetPseudoRandomGeneratorSeed(g, seed)
        self.lib.curandSetStream(g, ctypes.c_void_p(stream_ptr))
        return g

    def fill(self, g, name: str, ptr: int, n: int):
        L, p = self.lib, ctypes.c_void_p(ptr)
        if name == "bits_u32":
            st = L.curandGenerate(g, p, n)
        elif name == "uniform_f32":
            st = L.curandGenerateUniform(g, p, n)
        elif name == "uniform_f64":
            st = L.curandGenerateUniformDouble(g, p, n)
        elif name == "gaussian_f32":
            st = L.curandGenerateNormal(g, p, n, 0.0, 1.0)
        elif name == "gaussian_f64":
            st = L.curandGenerateNormalDouble(g, p, n, 0.0, 1.0)
        else:
            st = L.curandGenerateLogNormal(g, p, n, 0.0, 1.0)
        if st != 0:
            raise RuntimeError(f"cuRAND {name}: status {st}")

    def destroy(self, g):
        self.lib.curandDestroyGenerator(g)


# ----------------------------------------------------------------- oracle
def oracle_rate(seconds_per_case: float, cores: int, n_cap: int):
    """Oracle throughput on the host cores for each sweep case (bounded sample)."""
    import concurrent.futures as cf

    import oracle

    oracle.build()
    rates, detail = {}, {}
    chunk = 1 << 14
    for ek, en in ENGINES:
        for name, kind, dtype, p0, p1 in W.SWEEP_DISTS:
            t0 = time.perf_counter()
            done = 0
            futs = []
            with cf.ThreadPoolExecutor(max_workers=cores) as ex:
                idx = 0
                while time.perf_counter() - t0 < seconds_per_case and done < n_cap:
                    futs = [ex.submit(oracle.generate, ek, W.SWEEP_SEED,
                                      oracle.words_for(kind, dtype, (idx + i) * chunk), kind,
                                      dtype, p0, p1, chunk) for i in range(cores)]
                    for f in futs:
                        f.result()
                    idx += cores
                    done += cores * chunk
            dt = time.perf_counter() - t0
            rates[f"{en}/{name}"] = done / dt
            detail[f"{en}/{name}"] = {"samples": done, "seconds": round(dt, 3)}
    return rates, detail


# 32x32 products per output sample, counted from the algorithms as
# implemented: Philox4x32-10 is 20 products per 4-word block; an MRG32k3a word
# is 7 (per component two multiplier products, then the folds of 2^32 = c
# mod m: one 32-bit product for m1, one wide and one 32-bit product for m2);
# the fixed-point FP64 Box-Muller pair is 35 products (log: 7, square root:
# 6, sine and cosine: 16, the two final products: 6) on top of the products
# of its 4 words.
BM64_PRODUCTS_PER_PAIR = 35

# DRAM bytes (read + write) per launch at n = 10^9 from ncu captures of the
# current kernels: one launch of 2.68e8 samples scaled by 1e9 / 2.68e8;
# a kernel whose code changed after its capture is left out (no number
# rather than a stale one).
NCU_TRAFFIC_PER_1E9 = {
    "mrg32k3a/gaussian_f64": (2.083313e9 + 0.118e6) / 0.268,
    "philox4x32_10/gaussian_f64": (2.082409e9 + 0.304e6) / 0.268,
    "philox4x32_10/uniform_f32": (1.010023e9 + 0.042e6) / 0.268,
    "philox4x32_10/uniform_f64": (2.081978e9 + 0.056e6) / 0.268,
}

# The method's own 32x32 -> 64-bit products per sample, independent of how
# the kernels implement the arithmetic around them: two multiplier products
# per Philox4x32-10 round, ten rounds per 4-word block (5 per word); two
# multiplier products per MRG32k3a component step (4 per word; the modular
# reductions are counted only in the implementation figures above).
METHOD_PRODUCTS_PER_WORD = {"philox4x32_10": 5, "mrg32k3a": 4}
WORDS_PER_SAMPLE = {"bits_u32": 1, "uniform_f32": 1, "uniform_f64": 2, "gaussian_f32": 1,
                    "gaussian_f64": 2, "lognormal_f32": 1}

# Method-level transcendental operations, evaluated by CUDA's math library in
# the op-rate probes (csrc/probes.cu); samples/s a fill could reach if those
# operations were its only work.  FP64 ones are context: the library computes
# them in integer fixed point, off the FP64 pipe.
OP_KINDS = {"fp32_box_muller_pair": 0, "fp32_expf": 1, "fp32_normcdfinvf": 2,
            "fp64_box_muller_pair": 3, "fp64_fma": 4, "fp32_fma": 5, "xu_lg2_approx": 6,
            "fp64_normcdfinv": 7}


def transcendental_ceiling(name: str, ops: dict):
    """(samples/s, what) of the method's transcendental operations, or None."""
    if name == "gaussian_f32":
        return 2 * ops["fp32_box_muller_pair"], "CUDA logf + sincospif + sqrtf per pair"
    if name == "lognormal_f32":
        t = 0.5 / ops["fp32_box_muller_pair"] + 1.0 / ops["fp32_expf"]
        return 1.0 / t, "CUDA logf + sincospif + sqrtf per pair, expf per sample"
    if name == "icdf_gaussian_f32":
        return ops["fp32_normcdfinvf"], "CUDA normcdfinvf per sample"
    if name == "icdf_lognormal_f32":
        return 1.0 / (1.0 / ops["fp32_normcdfinvf"] + 1.0 / ops["fp32_expf"]), \
            "CUDA normcdfinvf + expf per sample"
    return None
PRODUCTS_PER_SAMPLE = {
    "philox4x32_10/bits_u32": 5, "philox4x32_10/uniform_f32": 5,
    "philox4x32_10/uniform_f64": 10, "philox4x32_10/gaussian_f32": 5,
    "philox4x32_10/gaussian_f64": (20 + BM64_PRODUCTS_PER_PAIR) / 2,
    "philox4x32_10/lognormal_f32": 5,
    "mrg32k3a/bits_u32": 7, "mrg32k3a/uniform_f32": 7, "mrg32k3a/uniform_f64": 14,
    "mrg32k3a/gaussian_f32": 7, "mrg32k3a/gaussian_f64": (28 + BM64_PRODUCTS_PER_PAIR) / 2,
    "mrg32k3a/lognormal_f32": 7,
}


def probe_ceilings(buf_ptr: int, nbytes: int, sink_ptr: int):
    """Write-only bandwidth, the 32x32->64 product rate and the method-level
    operation rates (OP_KINDS) on this GPU."""
    path = os.path.join(ROOT, "paper_2109_01329_gb300", "libgrng_probes.so")
    lib = ctypes.CDLL(path)
    lib.grng_probe_op_rate.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]
    ops = {}
    for nm, k in OP_KINDS.items():
        r = ctypes.c_double()
        if lib.grng_probe_op_rate(ctypes.c_void_p(sink_ptr), k, ctypes.byref(r)) != 0:
            raise RuntimeError(f"op-rate probe {nm} failed")
        ops[nm] = r.value
    lib.grng_probe_write_gbs.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double)]
    lib.grng_probe_mulwide_rate.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    w, m = ctypes.c_double(), ctypes.c_double()
    if lib.grng_probe_write_gbs(ctypes.c_void_p(buf_ptr), nbytes, 5, ctypes.byref(w)) != 0:
        raise RuntimeError("write probe failed")
    if lib.grng_probe_mulwide_rate(ctypes.c_void_p(sink_ptr), ctypes.byref(m)) != 0:
        raise RuntimeError("multiply probe failed")
    return w.value, m.value, ops


def aggregate_rate(rates: dict, n: int) -> float:
    """Samples/s for the whole sweep step (n samples per case) at per-case rates."""
    total_t = sum(n / r for r in rates.values())
    return len(rates) * n / total_t


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q / 100.0 * (len(xs) - 1))))]


# Fills outside the config-2 sweep, timed the same way: the inverse-CDF methods,
# FP64 lognormal, the affine FP64 gaussian and a general FP32 range.
EXTRA_DISTS = [
    ("icdf_gaussian_f32", 4, 1, 0.0, 1.0), ("icdf_lognormal_f32", 5, 1, 0.0, 1.0),
    ("icdf_gaussian_f64", 4, 2, 0.0, 1.0), ("lognormal_f64", 3, 2, 0.0, 1.0),
    ("gaussian_f64_m3_s0.25", 2, 2, -3.0, 0.25), ("uniform_f32_2_5", 1, 1, 2.0, 5.0),
    ("uniform_f64_2_5", 1, 2, 2.0, 5.0),
]


def run_config1(grng, torch, dev, stream, reps=50):
    """2^20 FP32 uniforms on [0, 1) from Philox4x32-10, seed 0x12345678, offset 0
    (the bit-exact small case): device time per launch (CUDA events, median of
    reps) and host time per call (launch overhead included)."""
    n = 1 << 20
    out = torch.empty(n, dtype=torch.float32, device=dev)
    d = grng.Distribution.uniform(0.0, 1.0, grng.F32)
    e = grng.Engine(0, 0x12345678, 0)
    with torch.cuda.stream(stream):
        for _ in range(5):
            grng.generate(d, e, out, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            grng.generate(d, e, out, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        host = []
        for _ in range(reps):
            t0 = time.perf_counter()
            grng.generate(d, e, out, stream=stream)
            host.append(time.perf_counter() - t0)
        torch.cuda.synchronize()
        # ten launches captured in a CUDA graph: the kernel's own time at this
        # size, without the host's per-call work between launches
        # (captured on a stream of its own: capture needs a non-default stream)
        g10 = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(stream)
        with torch.cuda.graph(g10, stream=cap):
            for _ in range(10):
                grng.generate(d, e, out, stream=cap)
        stream.wait_stream(cap)
        g10.replay()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for a, b in gev:
            a.record(stream)
            g10.replay()
            b.record(stream)
        torch.cuda.synchronize()
        del g10
    ms_graph = statistics.median(a.elapsed_time(b) for a, b in gev) / 10
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    return {"workload": "Philox4x32-10 seed 0x12345678 offset 0: 2^20 FP32 uniforms [0,1)",
            "device_us": round(ms * 1e3, 2), "gsamples_s": round(n / ms / 1e6, 2),
            "write_gbs": round(4 * n / ms / 1e6, 1),
            "host_call_us": round(statistics.median(host) * 1e6, 2), "reps": reps,
            "graph_device_us_per_launch": round(ms_graph * 1e3, 2),
            "graph_gsamples_s": round(n / ms_graph / 1e6, 2),
            "note": "4 MB: launch and ramp-up bound, far below the HBM roofline; device_us "
                    "includes the gap while the host issues the call, graph_* do not"}


def run_config3(grng, torch, dev, stream, hbm_peak, reps=3):
    """16384 substreams x 65536 FP64 gaussians (0, 1) in one launch per engine:
    MRG32k3a substreams 2^76 words apart, Philox4x32-10 substreams 2^40 words
    apart, seed 2021 (2^30 doubles = 8.6 GB per launch)."""
    ns, per = 16384, 65536
    out = torch.empty(ns * per, dtype=torch.float64, device=dev)
    d = grng.Distribution.gaussian(0.0, 1.0, grng.F64)
    res = {"workload": "16384 substreams x 65536 FP64 gaussians (0,1), seed 2021, one launch "
                       "per engine (MRG32k3a stride 2^76, Philox4x32-10 stride 2^40)"}
    for ek, en, stride in ((1, "mrg32k3a", 1 << 76), (0, "philox4x32_10", 1 << 40)):
        e = grng.Engine(ek, W.SWEEP_SEED, 0)
        with torch.cuda.stream(stream):
            grng.generate_substreams(d, e, out, per, ns, stride, stream=stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            for a, b in ev:
                a.record(stream)
                grng.generate_substreams(d, e, out, per, ns, stride, stream=stream)
                b.record(stream)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        gbs = 8 * ns * per / ms / 1e6
        res[en] = {"ms": round(ms, 3), "gsamples_s": round(ns * per / ms / 1e6, 2),
                   "write_gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4)}
    del out
    return res


def _event_ms(torch, stream, fn, reps):
    """Median CUDA-event time of fn() on stream after one untimed call."""
    with torch.cuda.stream(stream):
        fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def run_offset_paths(grng, torch, dev, n, buf, stream, reps=3):
    """Fills whose output start or word phase does not line up with 16-byte
    groups, each beside the same fill lined up: a Box-Muller pair split by the
    pointer (output at element offset 1), substreams of odd length at a word
    stride that is not a multiple of 4, and the 4096-request batch with every
    output at element offset 1."""
    res = {}
    for ek, en in ENGINES:
        for name, kind, dtype in (("gaussian_f32", 2, 1), ("gaussian_f64", 2, 2)):
            es = 8 if dtype == 2 else 4
            tdt = torch.float32 if dtype == 1 else torch.float64
            whole = buf[: (n + 2) * es].view(tdt)
            d = grng.Distribution(kind, dtype, 0.0, 1.0)
            times = {}
            for label, out in (("aligned", whole[:n]), ("pointer_plus_1", whole[1:n + 1])):
                e = grng.Engine(ek, W.SWEEP_SEED, 0)
                times[label] = _event_ms(torch, stream,
                                         lambda: grng.generate(d, e, out, stream=stream), reps)
            res[f"{en}/{name}"] = {k: round(v, 4) for k, v in times.items()}
            res[f"{en}/{name}"]["ratio"] = round(times["pointer_plus_1"] / times["aligned"], 3)
    # substreams: 16384 x 65536 FP32 gaussians, stride 2^40, against
    # 16384 x 65537 at stride 2^40 + 1 (every stream at its own phase)
    d = grng.Distribution(2, 1, 0.0, 1.0)
    for ek, en in ENGINES:
        times = {}
        for label, per, stride in (("aligned", 65536, 1 << 40), ("odd_len_odd_stride", 65537,
                                                                  (1 << 40) + 1)):
            out = buf[: 16384 * per * 4].view(torch.float32)
            e = grng.Engine(ek, W.SWEEP_SEED, 0)
            times[label] = _event_ms(torch, stream, lambda: grng.generate_substreams(
                d, e, out, per, 16384, stride, stream=stream), reps)
        res[f"{en}/substreams_gaussian_f32"] = {k: round(v, 4) for k, v in times.items()}
        res[f"{en}/substreams_gaussian_f32"]["ratio"] = round(
            times["odd_len_odd_stride"] / times["aligned"], 3)
    # one stream at word offsets 1, 2, 3 (the groups straddle counter blocks or
    # MRG32k3a units), a fresh engine per call
    for ek, en in ENGINES:
        for name, kind, dtype, p0, p1 in (("bits", 0, 0, 0.0, 0.0), ("uniform_f32", 1, 1, 0.0, 1.0)):
            out = buf[: n * 4].view(torch.int32 if dtype == 0 else torch.float32)
            d = grng.Distribution(kind, dtype, p0, p1)
            times = {}
            for off in (0, 1, 2, 3):
                times[f"word_offset_{off}"] = _event_ms(
                    torch, stream, lambda: grng.generate(d, grng.Engine(ek, W.SWEEP_SEED, off),
                                                         out, stream=stream), reps)
            key = f"{en}/{name}_word_offsets"
            res[key] = {k: round(v, 4) for k, v in times.items()}
            res[key]["worst_ratio"] = round(
                max(times[f"word_offset_{o}"] for o in (1, 2, 3)) / times["word_offset_0"], 3)
    # the batched table, outputs at element offset 0 and 1
    table = W.batched_requests(4096)
    tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}
    times = {}
    for label, shift in (("aligned", 0), ("pointer_plus_1", 1)):
        reqs = []
        for q in table:
            nm, kind, dtype, p0, p1 = q["dist"]
            o = torch.empty(q["n"] + shift, dtype=tdt[dtype], device=dev)[shift:]
            reqs.append((grng.Engine(0, q["seed"], 0), grng.Distribution(kind, dtype, p0, p1), o,
                         q["n"]))
        b = grng.Batch(reqs, ipt=8, stream=stream)
        b.autotune(stream=stream)
        times[label] = _event_ms(torch, stream, lambda: b.launch(stream=stream), 10)
        del b, reqs
    res["batched_4096"] = {k: round(v, 4) for k, v in times.items()}
    res["batched_4096"]["ratio"] = round(times["pointer_plus_1"] / times["aligned"], 3)
    return res


def run_extra(grng, torch, dev, n, buf, stream, reps, hbm_peak):
    out = {}
    tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}
    for ek, en in ENGINES:
        for name, kind, dtype, p0, p1 in EXTRA_DISTS:
            es = 8 if dtype == 2 else 4
            view = buf[: n * es].view(tdt[dtype])
            d = grng.Distribution(kind, dtype, p0, p1)
            e = grng.Engine(ek, W.SWEEP_SEED, 0)
            with torch.cuda.stream(stream):
                grng.generate(d, e, view, stream=stream)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps)]
                for a, b in ev:
                    a.record(stream)
                    grng.generate(d, e, view, stream=stream)
                    b.record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in ev)
            gbs = n * es / (ms * 1e-3) / 1e9
            out[f"{en}/{name}"] = {"ms": round(ms, 4), "gsamples_s": round(n / ms / 1e6, 2),
                                   "write_gbs": round(gbs, 1),
                                   "frac_hbm": round(gbs / hbm_peak, 4)}
    return out


def run_tts(grng, torch, dev, stream, with_curand, sizes=(10**3, 10**6, 10**8), reps=7):
    """Time to solution of one call, as the paper's RNG burner counts it
    (Sec. 7): engine or generator creation, seeding, one fill of n FP32
    uniforms on [0,1) and a stream synchronisation, host wall clock, median of
    reps after one untimed call; ours against cuRAND's host API (create, seed,
    set stream, generate, sync, destroy), both engines."""
    out = torch.empty(max(sizes), dtype=torch.float32, device=dev)
    cr = None
    if with_curand:
        try:
            cr = Curand()
        except Exception:  # noqa: BLE001
            cr = None
    d = grng.Distribution.uniform(0.0, 1.0)
    res = {}
    for ek, en in ENGINES:
        res[en] = {}
        for n in sizes:
            def ours():
                e = grng.Engine(ek, W.SWEEP_SEED, 0)
                grng.generate(d, e, out, n=n, stream=stream)
                stream.synchronize()

            def theirs():
                g = cr.generator(ek, W.SWEEP_SEED, stream.cuda_stream)
                cr.fill(g, "uniform_f32", out.data_ptr(), n)
                stream.synchronize()
                cr.destroy(g)

            row = {}
            for key, fn in (("ours_us", ours), ("curand_us", theirs if cr else None)):
                if fn is None:
                    continue
                fn()
                ts = []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    fn()
                    ts.append(time.perf_counter() - t0)
                row[key] = round(statistics.median(ts) * 1e6, 1)
            if "curand_us" in row:
                row["speedup_ours"] = round(row["curand_us"] / row["ours_us"], 2)
            res[en][str(n)] = row
    return {"how": "create + seed + one FP32 uniform fill of n + stream sync, host wall clock, "
                   f"median of {reps}", **res}


def run_batched(grng, torch, dev, reps):
    """Batched requests: 4096 Philox engines (seeds 1..4096), log-uniform sizes in
    [64, 2^20], five distributions; one graph-replayed persistent launch vs
    one grng_generate launch per request (back to back on one stream), both
    called eagerly and replayed from a CUDA graph of the 4096 launches."""
    table = W.batched_requests(4096)
    tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}
    reqs, total = [], 0
    for q in table:
        name, kind, dtype, p0, p1 = q["dist"]
        out = torch.empty(q["n"], dtype=tdt[dtype], device=dev)
        reqs.append((grng.Engine(0, q["seed"], 0), grng.Distribution(kind, dtype, p0, p1), out,
                     q["n"]))
        total += q["n"]
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        # per-request launches: each request is its own grng_generate call
        def loop():
            for e, d, o, n in reqs:
                grng.generate(d, e, o, n=n, stream=stream)
        for _ in range(3):
            loop()
        loop_ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            loop()
            e1.record(stream)
            e1.synchronize()
            loop_ms.append(e0.elapsed_time(e1))
        # the same per-request launches captured once into a CUDA graph: no host
        # work per request on replay (the stronger baseline: only the GPU-side
        # cost of 4096 small launches remains)
        g_loop = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_loop, stream=stream):
            loop()
        for _ in range(3):
            g_loop.replay()
        loop_graph_ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g_loop.replay()
            e1.record(stream)
            e1.synchronize()
            loop_graph_ms.append(e0.elapsed_time(e1))
        del g_loop
        b = grng.Batch(reqs, ipt=8, stream=stream)
        ipt, ctas, tune_ms = b.autotune(stream=stream)
        b.launch(stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            b.launch(stream=stream)
        for _ in range(3):
            graph.replay()
        batch_ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            batch_ms.append(e0.elapsed_time(e1))
    med_loop, med_batch = statistics.median(loop_ms), statistics.median(batch_ms)
    out_bytes = sum(o.numel() * o.element_size() for _, _, o, _ in reqs)
    return {"workload": "4096 Philox engines (seeds 1..4096), n log-uniform in [64, 2^20], "
                        "distribution uniform over {bits u32, uniform f32 [0,1), gaussian f32, "
                        "lognormal f32, uniform f64 [-1,1)}, numpy PCG64 seed 2021",
            "requests": len(reqs), "samples": total, "bytes": out_bytes,
            "per_request_ms_p50": round(med_loop, 4), "per_request_ms_p99": round(_pct(loop_ms, 99), 4),
            "batched_graph_ms_p50": round(med_batch, 4),
            "batched_graph_ms_p99": round(_pct(batch_ms, 99), 4),
            "speedup": round(med_loop / med_batch, 3),
            "per_request_graph_ms_p50": round(statistics.median(loop_graph_ms), 4),
            "speedup_vs_per_request_graph": round(statistics.median(loop_graph_ms) / med_batch, 3),
            "batched_gsamples_s": round(total / med_batch / 1e6, 2),
            "batched_write_gbs": round(out_bytes / med_batch / 1e6, 1),
            "per_request_gsamples_s": round(total / med_loop / 1e6, 2),
            "autotune": {"ipt": ipt, "ctas_per_sm": ctas, "ms": round(tune_ms, 4),
                         "searched": "ipt {1,2,4,8,16,32} x CTAs/SM {1,2,4,6,8,12,16}"},
            "reps": reps}


def run_serving(grng, torch, dev, seconds, stress, hold):
    """FastCaloSim-shaped serving.  Poisson arrivals at 2000 events/s,
    hits ~ lognormal(mean 8000, sigma 0.8) clipped to [100, 200000]; each event
    = 3h FP32 uniforms + h FP32 gaussians from its own Philox engine (seed =
    event id); 4 GB admission budget; replayed in real time, then compressed
    `stress` times so that the budget and the backlog bind."""
    t, hits = W.fastcalosim_events(rate_hz=2000.0, duration_s=seconds, seed=2021)
    u = grng.Distribution.uniform(0.0, 1.0, grng.F32)
    z = grng.Distribution.gaussian(0.0, 1.0, grng.F32)
    reqs = [grng.serve_request(i + 1, [(u, 3 * int(h)), (z, int(h))]) for i, h in enumerate(hits)]
    out = {"workload": f"Poisson 2000 events/s for {seconds:g} s ({len(reqs)} events), hits "
                       "lognormal mean 8000 sigma 0.8 clipped [100, 2e5], 3h uniform f32 + h "
                       "gaussian f32 per event from Philox seed = event id, 4 GB budget, "
                       "3 stream slots",
           "events": len(reqs), "samples": int(4 * hits.sum())}
    srv = grng.Server(4 << 30, num_streams=3, auto_release=True, device=dev)
    # real time; then compressed `stress` times with every output held for
    # `hold` seconds after completion (a consumer that keeps each event's
    # numbers that long), so that the 4 GB budget binds and admission waits;
    # the burst (every event at once) lasts a few tens of milliseconds, so it
    # is replayed five times and the median run is reported
    for name, scale, runs, hold_s in (("real_time", 1.0, 1, 0.0),
                                      (f"stress_{stress:g}x_hold_{hold:g}s", 1.0 / stress, 1, hold),
                                      ("burst", 1e-9, 5, 0.0)):
        results = []
        srv.set_release_delay(hold_s)
        for _ in range(runs):
            srv.reset_stats()
            srv.replay(t, reqs, time_scale=scale)
            srv.drain(timeout_s=600)
            if hold_s > 0:
                time.sleep(hold_s + 0.2)  # the held outputs go back to the budget
            st = srv.stats()
            results.append({
                "gsamples_s": round(st["samples"] / st["wall_s"] / 1e9, 3) if st["wall_s"]
                else None,
                "latency_p50_us": round(st["latency_p50_us"], 1),
                "latency_p99_us": round(st["latency_p99_us"], 1),
                "latency_max_us": round(st["latency_max_us"], 1),
                "completed": st["completed"], "rejected": st["rejected"],
                "batches": st["batches"],
                "mean_batch_events": round(st["mean_batch_requests"], 2),
                "peak_pool_gb": round(st["peak_pool_bytes"] / 1e9, 3),
                "admit_wait_p50_us": round(st["admit_wait_p50_us"], 1),
                "admit_wait_p99_us": round(st["admit_wait_p99_us"], 1),
                "wall_s": round(st["wall_s"], 3)})
        results.sort(key=lambda r: r["gsamples_s"] or 0.0)
        out[name] = dict(results[len(results) // 2])
        if runs > 1:
            out[name]["runs_gsamples_s"] = [r["gsamples_s"] for r in results]
    srv.close()
    # the plain form: two grng_generate launches per event, back to back on one
    # stream, into one preallocated buffer (no admission, no batching)
    buf = torch.empty(int(4 * hits.max()), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for i, h in enumerate(hits):
            h = int(h)
            e = grng.Engine(0, i + 1, 0)
            grng.generate(u, e, buf[:3 * h], stream=stream)
            grng.generate(z, e, buf[3 * h:4 * h], stream=stream)
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - t0
    out["per_event_launches"] = {"gsamples_s": round(out["samples"] / wall / 1e9, 3),
                                 "wall_s": round(wall, 3), "gpu_ms": round(e0.elapsed_time(e1), 3)}
    if out["burst"]["gsamples_s"]:
        out["burst_speedup_vs_per_event"] = round(out["burst"]["gsamples_s"] /
                                                  out["per_event_launches"]["gsamples_s"], 2)
    return out


def sweep_config(n: int, world: int) -> dict:
    """The workload both arms report: the config-2 fill sweep."""
    return {"workload": f"fill sweep n={n:.0e} per GPU: Philox4x32-10 and MRG32k3a x "
                        "{bits u32, uniform f32 [0,1), uniform f64 [0,1), gaussian "
                        "f32 (0,1), gaussian f64 (0,1), lognormal f32 (0,1)}, "
                        "seed 2021",
            "n_per_fill": n, "fills_per_step": len(ENGINES) * len(W.SWEEP_DISTS),
            "parallelism": f"shard{world} (rank r fills words from r * words_for(n))",
            "l2": "every fill writes 4-8 GB, larger than the 129 MB L2"}


def _long_double_note() -> str:
    """How the oracle's long double arithmetic runs on this host."""
    import platform

    m = platform.machine()
    if m in ("aarch64", "arm64"):
        return ("the oracle evaluates Box-Muller and the inverse CDF in long double, which on "
                "this aarch64 host is IEEE binary128 in software (so its gaussian and lognormal "
                "cases run about 20x slower than its uniforms)")
    return f"the oracle evaluates Box-Muller and the inverse CDF in long double ({m} host)"


def run_reference(args):
    """The oracle as the reference arm: bounded samples of the sweep per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import concurrent.futures as cf

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    per_case = args.ref_samples
    chunk = max(1, per_case // cores)

    def step():
        for ek, _ in ENGINES:
            for name, kind, dtype, p0, p1 in W.SWEEP_DISTS:
                with cf.ThreadPoolExecutor(max_workers=cores) as ex:
                    list(ex.map(lambda i: oracle.generate(
                        ek, W.SWEEP_SEED, oracle.words_for(kind, dtype, i * chunk), kind, dtype,
                        p0, p1, chunk), range(cores)))

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    samples = args.steps * len(ENGINES) * len(W.SWEEP_DISTS) * chunk * cores
    value = samples / dt / 1e9
    sample_desc = (f"{chunk * cores} samples per (engine, distribution) case per step, "
                   f"{len(ENGINES) * len(W.SWEEP_DISTS)} cases, seed 2021, split over {cores} "
                   "threads by word offset; " + _long_double_note())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/f32/f64", "data": "synthetic",
            "config": sweep_config(int(args.n), args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample_desc + "; the rate stands for the sweep's "
                                                     "samples/s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ours
def run_ours(args):
    import torch

    import paper_2109_01329_gb300 as grng
    from paper_2109_01329_gb300 import build as gbuild
    from paper_2109_01329_gb300 import shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world and world > 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        gbuild.build()
    if world > 1:
        dist.barrier()
    grng.load()

    n = int(args.n)
    hbm_peak, peak_src = _peaks()
    stream = torch.cuda.current_stream(dev)
    buf = torch.empty(n * 8 + 256, dtype=torch.uint8, device=dev)  # + room for offset outputs
    tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}
    cases = [(ek, en, d) for ek, en in ENGINES for d in W.SWEEP_DISTS]
    if args.only:
        cases = [c for c in cases if f"{c[1]}/{c[2][0]}" in args.only.split(",")]
        if not cases:
            raise SystemExit(f"--only {args.only}: no such case")
    # weak scaling: rank r fills the r-th block of n outputs of one long stream
    def rank_offset(kind, dtype):
        return grng.words_for(grng.Distribution(kind, dtype, 0.0, 1.0), n) * rank

    def one_step(events=None):
        for i, (ek, en, (name, kind, dtype, p0, p1)) in enumerate(cases):
            es = 8 if dtype == 2 else 4
            out = buf[: n * es].view(tdt[dtype])
            e = grng.Engine(ek, W.SWEEP_SEED, rank_offset(kind, dtype))
            if events is not None:
                events[i][0].record(stream)
            grng.generate(grng.Distribution(kind, dtype, p0, p1), e, out)
            if events is not None:
                events[i][1].record(stream)

    # launch geometry per fill from the library's autotuner (the outputs do not
    # depend on it); the choice is reported per kernel
    geometry = {}
    for ek, en, (name, kind, dtype, p0, p1) in cases:
        d = grng.Distribution(kind, dtype, p0, p1)
        es = 8 if dtype == 2 else 4
        gm = {"chosen": None}
        if not args.no_tune:
            _, t_best, t_builtin = grng.fill_autotune(ek, d, buf[: n * es].view(tdt[dtype]), n,
                                                      stream=stream)
            gm = {"tuned_ms": round(t_best, 4), "builtin_ms": round(t_builtin, 4)}
        gm["chosen"] = grng.fill_geometry(ek, d, n)
        geometry[f"{en}/{name}"] = gm
    for _ in range(max(args.warmup, 0)):
        one_step()
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in cases] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        one_step(ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    samples_per_step = n * len(cases) * world
    value = samples_per_step / (ms_per_step * 1e-3) / 1e9

    # ceilings measured live on this GPU (outside the timed region)
    sink = torch.zeros(16, dtype=torch.int32, device=dev)
    write_gbs, mul_probe, ops = probe_ceilings(buf.data_ptr(), buf.numel(), sink.data_ptr())
    # integer roofline peak from unit counts and the clock: per SM 4 sub-partitions
    # x 16 lanes of the FMA-heavy pipe, a 32x32->64 product taking two passes,
    # i.e. 32 products per clock per SM, at the median SM clock under load
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_hz = (clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0) * 1e6
    mul_rate = n_sms * 32 * sm_hz
    per_kernel = {}
    for i, (ek, en, (name, kind, dtype, p0, p1)) in enumerate(cases):
        key = f"{en}/{name}"
        ms = statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
        es = 8 if dtype == 2 else 4
        rate = n / (ms * 1e-3)
        gbs = n * es / (ms * 1e-3) / 1e9
        prods = PRODUCTS_PER_SAMPLE[key] * n
        tops = prods / (ms * 1e-3) / 1e12
        m_prods = METHOD_PRODUCTS_PER_WORD[en] * WORDS_PER_SAMPLE[name]
        # ceilings in samples/s: the roofline of the target statement is the
        # slower of output bytes at HBM bandwidth and integer operations at
        # peak (the products as implemented); the method view counts only the
        # method's own products; FP32 transcendental fills add the rate of
        # their method operations in CUDA's math library
        ceil = {"hbm_write": hbm_peak * 1e9 / es, "int_impl": mul_rate / PRODUCTS_PER_SAMPLE[key],
                "int_method": mul_rate / m_prods}
        tc = transcendental_ceiling(name, ops)
        if tc is not None:
            ceil["transcendental"] = tc[0]
        impl_keys = [c for c in ceil if c != "int_method"]
        meth_keys = [c for c in ceil if c != "int_impl"]
        bound = min(impl_keys, key=ceil.get)
        bound_m = min(meth_keys, key=ceil.get)
        per_kernel[key] = {"ms": round(ms, 4), "gsamples_s": round(rate / 1e9, 2),
                           "write_gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4),
                           "frac_write_probe": round(gbs / write_gbs, 4),
                           "products_per_launch": prods, "tproducts_s": round(tops, 3),
                           "frac_int": round(tops * 1e12 / mul_rate, 4),
                           "frac_int_method": round(rate * m_prods / mul_rate, 4),
                           "ceilings_gsamples_s": {c: round(v / 1e9, 2) for c, v in ceil.items()},
                           "bound": "hbm" if bound == "hbm_write" else "alu",
                           "bound_ceiling": bound,
                           "frac_roofline": round(rate / ceil[bound], 4),
                           "bound_ceiling_method": bound_m,
                           "frac_roofline_method": round(rate / ceil[bound_m], 4)}
        if tc is not None:
            per_kernel[key]["transcendental_ops"] = tc[1]
        per_kernel[key]["geometry"] = geometry[key]
        if name == "gaussian_f64":
            # context: the method's FP64 operations in CUDA's FP64 math library
            per_kernel[key]["vs_fp64_libm_rate"] = round(
                rate / (2 * ops["fp64_box_muller_pair"]), 2)
    dom_name = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dom = per_kernel[dom_name]
    traffic = args.traffic
    if traffic is None and dom_name in NCU_TRAFFIC_PER_1E9:
        traffic = round(NCU_TRAFFIC_PER_1E9[dom_name] * n / 1e9)
    if dom["bound_ceiling"] == "hbm_write":
        roofline = {"kernel": dom_name, "bound": "hbm", "achieved": dom["write_gbs"],
                    "peak": hbm_peak, "unit": "GB/s", "frac": dom["frac_hbm"],
                    "traffic": traffic, "peak_source": f"{peak_src} hbm_gbs (copy)",
                    "bytes_per_launch": n * (8 if "f64" in dom_name else 4)}
    elif dom["bound_ceiling"] == "int_impl":
        roofline = {"kernel": dom_name, "bound": "alu", "achieved": dom["tproducts_s"],
                    "peak": round(mul_rate / 1e12, 3), "unit": "T products/s (32x32->64)",
                    "frac": dom["frac_int"], "traffic": traffic,
                    "peak_source": f"derived: {n_sms} SMs x 32 products/clock x "
                                   f"{sm_hz / 1e6:.0f} MHz (a live independent-chain probe "
                                   f"reaches {mul_probe / 1e12:.2f} T/s)",
                    "products_per_launch": dom["products_per_launch"],
                    "bytes_per_launch": n * (8 if "f64" in dom_name else 4)}
    else:
        roofline = {"kernel": dom_name, "bound": "alu", "achieved": dom["gsamples_s"],
                    "peak": dom["ceilings_gsamples_s"]["transcendental"], "unit": "Gsamples/s",
                    "frac": dom["frac_roofline"], "traffic": traffic,
                    "peak_source": "live probe: " + dom["transcendental_ops"],
                    "bytes_per_launch": n * (8 if "f64" in dom_name else 4)}
    roofline["method_view"] = {"bound_ceiling": dom["bound_ceiling_method"],
                               "frac": dom["frac_roofline_method"],
                               "ceilings_gsamples_s": dom["ceilings_gsamples_s"]}
    target = per_kernel.get("philox4x32_10/uniform_f32", dom)
    # the target statement's headline: Philox FP32 uniform fill at >= 0.80 of
    # its roofline (HBM write bound), against the copy peak and the live
    # write-only probe
    roofline["target_batched_vs_per_request"] = None  # filled below when the batch runs
    roofline["target_philox_uniform_f32"] = {
        "write_gbs": target["write_gbs"], "frac": target["frac_roofline"],
        "frac_hbm_copy_peak": target["frac_hbm"],
        "frac_write_only_probe": target["frac_write_probe"],
        "write_only_probe_gbs": round(write_gbs, 1), "meets_0_80": target["frac_roofline"] >= 0.80,
        "bytes_per_launch": n * 4,
        "traffic": (round(NCU_TRAFFIC_PER_1E9["philox4x32_10/uniform_f32"] * n / 1e9)
                    if "philox4x32_10/uniform_f32" in per_kernel else None)}

    # cuRAND on the same fills (generate calls only; generator created outside)
    curand = None
    if not args.skip_curand and rank == 0:
        try:
            cr = Curand()
            curand = {}
            for ek, en, (name, kind, dtype, p0, p1) in cases:
                es = 8 if dtype == 2 else 4
                gen = cr.generator(ek, W.SWEEP_SEED, stream.cuda_stream)
                for _ in range(2):
                    cr.fill(gen, name, buf.data_ptr(), n)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 3
                e0.record(stream)
                for _ in range(reps):
                    cr.fill(gen, name, buf.data_ptr(), n)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                cr.destroy(gen)
                ours = per_kernel[f"{en}/{name}"]["ms"]
                curand[f"{en}/{name}"] = {"ms": round(ms, 4), "gsamples_s": round(n / ms / 1e6, 2),
                                          "speedup_ours": round(ms / ours, 3)}
            tot_c = sum(v["ms"] for v in curand.values())
            curand["_step_ms"] = round(tot_c, 3)
            curand["_step_speedup_ours"] = round(tot_c / sum(v["ms"] for v in per_kernel.values()),
                                                 3)
        except Exception as ex:  # noqa: BLE001
            curand = {"unavailable": str(ex)[:200]}

    tts = None
    if rank == 0 and not args.skip_tts:
        tts = run_tts(grng, torch, dev, stream, not args.skip_curand)

    # end to end through the C ABI with host buffers (generate + D2H per chunk)
    e2e = None
    if not args.skip_e2e:
        host = torch.empty(n * 8, dtype=torch.uint8, pin_memory=True)
        work = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

        case_ms = {}

        def e2e_step():
            for ek, en, (name, kind, dtype, p0, p1) in cases:
                es = 8 if dtype == 2 else 4
                e = grng.Engine(ek, W.SWEEP_SEED, rank_offset(kind, dtype))
                tc = time.perf_counter()
                grng.generate_host(grng.Distribution(kind, dtype, p0, p1), e,
                                   host[: n * es].view(tdt[dtype]), work)
                case_ms[f"{en}/{name}"] = round((time.perf_counter() - tc) * 1e3, 2)

        e2e_step()
        # the host side of the link is shared with whatever else runs on the
        # machine, so several passes are timed and the median one reported
        step_s = []
        for _ in range(args.e2e_steps):
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            e2e_step()
            dt1 = time.perf_counter() - t0
            if world > 1:
                t = torch.tensor([dt1], device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                dt1 = float(t.item())
            step_s.append(dt1)
        dt = statistics.median(step_s)
        d2h = sum(n * (8 if d[2] == 2 else 4) for _, _, d in cases)
        # the device -> pinned host link alone: one 2 GiB copy, three times
        link_bytes = min(host.numel(), 2 << 30)
        src = torch.empty(link_bytes, dtype=torch.uint8, device=dev)
        host[:link_bytes].copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(3):
            host[:link_bytes].copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        link_gbs = 3 * link_bytes / (time.perf_counter() - t1) / 1e9
        del src
        e2e_gbs = d2h / dt / 1e9
        e2e = {"value": samples_per_step / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
               "ms_per_step": dt * 1e3, "passes_ms": [round(x * 1e3, 1) for x in step_s],
               "d2h_gbs": round(e2e_gbs, 1), "link_gbs": round(link_gbs, 1),
               "frac_link": round(e2e_gbs / link_gbs, 4), "per_case_ms": case_ms,
               "how": "grng_generate_host into pinned host memory, 256 MiB device staging, "
                      "host wall clock, median of the timed passes (per_case_ms: the last "
                      "pass); link_gbs is a plain 2 GiB device-to-pinned-host copy"}
        del host, work

    extra = None
    if rank == 0 and not args.skip_extra:
        extra = run_extra(grng, torch, dev, n, buf, stream, 3, hbm_peak)

    config1 = config3 = offset_paths = None
    if rank == 0 and not args.skip_configs:
        config1 = run_config1(grng, torch, dev, stream)
        config3 = run_config3(grng, torch, dev, stream, hbm_peak)
        offset_paths = run_offset_paths(grng, torch, dev, n, buf, stream)

    batched = None
    if rank == 0 and not args.skip_batched:
        batched = run_batched(grng, torch, dev, args.batch_reps)

    if batched is not None:
        roofline["target_batched_vs_per_request"] = {
            "speedup": batched["speedup"], "batched_graph_ms": batched["batched_graph_ms_p50"],
            "per_request_ms": batched["per_request_ms_p50"], "meets_5x": batched["speedup"] >= 5,
            "per_request_graph_ms": batched["per_request_graph_ms_p50"],
            "speedup_vs_per_request_graph": batched["speedup_vs_per_request_graph"]}

    serving = None
    if rank == 0 and args.serve_seconds > 0:
        serving = run_serving(grng, torch, dev, args.serve_seconds, args.serve_stress,
                              args.serve_hold)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        cores = os.cpu_count() or 1
        rates, detail = oracle_rate(args.cpu_seconds, cores, n_cap=n)
        cpu = {"value": aggregate_rate(rates, n) / 1e9, "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": f"about {args.cpu_seconds:g} s per (engine, distribution) case, "
                         f"chunks of 16384 samples over {cores} threads by word offset; rate "
                         "scaled to the sweep step (n per case); " + _long_double_note(),
               "per_case": {k: {"gsamples_s": round(rates[k] / 1e9, 6), **detail[k]}
                            for k in rates}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32/f64",
            "data": "synthetic",
            "config": sweep_config(n, world),
            "roofline": roofline,
            "target_philox_uniform_f32": {"write_gbs": target["write_gbs"],
                                          "frac": target["frac_hbm"],
                                          "frac_roofline": target["frac_roofline"],
                                          "gsamples_s": target["gsamples_s"]},
            "ceilings": {"hbm_copy_gbs": hbm_peak, "write_only_gbs": round(write_gbs, 1),
                         "products_per_s": mul_rate, "products_per_s_probe": mul_probe,
                         "op_rates_per_s": {k: round(v, 1) for k, v in ops.items()}},
            "per_kernel": per_kernel, "curand": curand, "tts": tts, "other_fills": extra,
            "config1_2pow20_uniform": config1, "config3_substreams": config3,
            "offset_paths": offset_paths,
            "batched": batched, "serving": serving,
            "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk, "gpu_launches": args.steps * len(cases)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=float, default=1e9)
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="timed end-to-end passes; the median one is reported")
    ap.add_argument("--cpu-seconds", type=float, default=1.5)
    ap.add_argument("--ref-samples", type=int, default=1 << 21)
    ap.add_argument("--only", default="",
                    help="comma-separated engine/distribution cases (profiling runs)")
    ap.add_argument("--skip-curand", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-tts", action="store_true",
                    help="skip the time-to-solution calls (create + seed + fill + sync)")
    ap.add_argument("--skip-configs", action="store_true",
                    help="skip the timed small case (2^20 uniforms) and the substream launches")
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the fills outside the sweep (inverse CDF, FP64 lognormal, ...)")
    ap.add_argument("--batch-reps", type=int, default=20)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="seconds of the arrival trace to replay in real time (0: skip)")
    ap.add_argument("--serve-stress", type=float, default=20.0)
    ap.add_argument("--serve-hold", type=float, default=1.0,
                    help="seconds each output is held after completion in the stress replay")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the built-in launch geometry instead of autotuning each fill")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
