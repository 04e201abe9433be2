// Ceiling probes for the roofline of the fill kernels (measurement only; not
// part of the generation path and not declared in grng.h).
//
//   grng_probe_write_gbs: write-only HBM bandwidth of a plain 16-byte store
//     kernel over a caller buffer (the memory ceiling of a fill, which only
//     writes).
//   grng_probe_mulwide_rate: 32x32 -> 64-bit products per second, the
//     operation that bounds Philox rounds, MRG32k3a steps and the fixed-point
//     FP64 Box-Muller.  Two chain shapes, the faster one counts: 8
//     independent chains by a constant multiplier (as in a Philox round), and
//     4 chains whose multiplier is the neighbouring chain's value.
//   grng_probe_op_rate: operations per second of one of the method-level
//     operations below, evaluated with CUDA's own math library on inputs from
//     a per-thread linear congruential sequence (one 32-bit multiply-add per
//     input), several independent chains per thread, every SM busy:
//       0  FP32 Box-Muller pair: sqrtf(-2 logf(u1)) times sincospif(2 u2)
//       1  FP32 expf
//       2  FP32 normcdfinvf (the inverse-CDF method's Phi^-1)
//       3  FP64 Box-Muller pair: sqrt(-2 log(u1)) times sincospi(2 u2)
//       4  FP64 fused multiply-add (the FP64 pipe alone)
//       5  FP32 fused multiply-add
//       6  special-function unit: lg2.approx.ftz.f32
//       7  FP64 normcdfinv
//     These are the ceilings of the transcendental fills: how fast this GPU's
//     math library evaluates the method's operations, without generating
//     words or writing memory.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

__global__ void __launch_bounds__(256) probe_store(uint4* out, int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n16; j += stride)
    out[j] = make_uint4((uint32_t)j, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(256) probe_mulwide(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 8u + (uint32_t)k + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint64_t p = (uint64_t)a[k] * 0xD2511F53u;
      a[k] = (uint32_t)(p >> 32) ^ (uint32_t)p;
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x ^= a[k];
  if (x == 0x9E3779B9u) sink[0] = x;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_mulwide_cross(uint32_t* sink, int iters,
                                                           uint32_t seed) {
  uint32_t a0 = seed + threadIdx.x, a1 = a0 * 3u + 1u, a2 = a0 * 5u + 7u, a3 = a0 * 9u + 3u;
  // 64 products per trip (16 rounds of 4), so the loop control is negligible
  for (int i = 0; i < iters / 8; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint64_t p0, p1, p2, p3;
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(a0), "r"(a1));
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p1) : "r"(a1), "r"(a2));
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p2) : "r"(a2), "r"(a3));
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p3) : "r"(a3), "r"(a0));
      a0 = (uint32_t)(p0 >> 32) ^ (uint32_t)p0;
      a1 = (uint32_t)(p1 >> 32) ^ (uint32_t)p1;
      a2 = (uint32_t)(p2 >> 32) ^ (uint32_t)p2;
      a3 = (uint32_t)(p3 >> 32) ^ (uint32_t)p3;
    }
  }
  if ((a0 ^ a1 ^ a2 ^ a3) == 0x9E3779B9u) sink[0] = a0;  // keeps the chains alive
}

__device__ __forceinline__ uint32_t lcg(uint32_t x) { return x * 1664525u + 1013904223u; }
__device__ __forceinline__ float u_open_f32(uint32_t x) {  // (0, 1]
  return (float)((x >> 8) + 1u) * 0x1p-24f;
}
__device__ __forceinline__ double u_open_f64(uint32_t x) {
  return (double)((x >> 8) + 1u) * 0x1p-24;
}

constexpr int kOpChains = 4;

// Each thread runs kOpChains independent chains for iters steps; every step
// is one operation of the kind (a pair for the Box-Muller kinds).
template <int K>
__global__ void __launch_bounds__(256) probe_op(float* sink, int iters, uint32_t seed) {
  uint32_t x[kOpChains];
  float accf[kOpChains];
  double accd[kOpChains];
#pragma unroll
  for (int k = 0; k < kOpChains; ++k) {
    x[k] = seed + (blockIdx.x * 256u + threadIdx.x) * 977u + (uint32_t)k * 131u;
    accf[k] = 0.f;
    accd[k] = 0.0;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kOpChains; ++k) {
      if constexpr (K != 4 && K != 5) x[k] = lcg(x[k]);
      if constexpr (K == 0) {
        const uint32_t y = lcg(x[k]);
        const float rho = sqrtf(-2.0f * logf(u_open_f32(x[k])));
        float s, c;
        sincospif(2.0f * ((float)(y >> 8) * 0x1p-24f), &s, &c);
        accf[k] += rho * c + rho * s;
      } else if constexpr (K == 1) {
        accf[k] += expf(u_open_f32(x[k]) * 8.0f - 4.0f);
      } else if constexpr (K == 2) {
        accf[k] += normcdfinvf(u_open_f32(x[k]) * 0.999999f);
      } else if constexpr (K == 3) {
        const uint32_t y = lcg(x[k]);
        const double rho = sqrt(-2.0 * log(u_open_f64(x[k])));
        double s, c;
        sincospi(2.0 * ((double)(y >> 8) * 0x1p-24), &s, &c);
        accd[k] += rho * c + rho * s;
      } else if constexpr (K == 4) {
        accd[k] = fma(accd[k], 0.999999999, 1e-9);
      } else if constexpr (K == 5) {
        accf[k] = fmaf(accf[k], 0.9999f, 1e-4f);
      } else if constexpr (K == 6) {
        float l;
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(u_open_f32(x[k])));
        accf[k] += l;
      } else {
        accd[k] += normcdfinv(u_open_f64(x[k]) * 0.999999);
      }
    }
  }
  float t = 0.f;
  double td = 0.0;
#pragma unroll
  for (int k = 0; k < kOpChains; ++k) {
    t += accf[k];
    td += accd[k];
  }
  if (t == 1234.5f || td == 1234.5) sink[0] = t + (float)td;  // keeps the chains alive
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int grng_probe_op_rate(void* dev_sink, int kind,
                                                                           double* per_s) {
  if (kind < 0 || kind > 7 || per_s == nullptr) return 1;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return 4;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // about a millisecond or more per launch at the expected rates
  static const int kIters[8] = {64, 128, 64, 8, 1024, 4096, 2048, 8};
  const int iters = kIters[kind];
  const int grid = sms * 8;
  float* sink = (float*)dev_sink;
  auto launch = [&](uint32_t seed) {
    switch (kind) {
      case 0: probe_op<0><<<grid, 256>>>(sink, iters, seed); break;
      case 1: probe_op<1><<<grid, 256>>>(sink, iters, seed); break;
      case 2: probe_op<2><<<grid, 256>>>(sink, iters, seed); break;
      case 3: probe_op<3><<<grid, 256>>>(sink, iters, seed); break;
      case 4: probe_op<4><<<grid, 256>>>(sink, iters, seed); break;
      case 5: probe_op<5><<<grid, 256>>>(sink, iters, seed); break;
      case 6: probe_op<6><<<grid, 256>>>(sink, iters, seed); break;
      default: probe_op<7><<<grid, 256>>>(sink, iters, seed); break;
    }
  };
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch(1u);
  const int reps = 3;
  cudaEventRecord(a);
  for (int i = 0; i < reps; ++i) launch(2u + (uint32_t)i);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *per_s = (double)grid * 256.0 * iters * kOpChains * reps / (ms * 1e-3);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

extern "C" __attribute__((visibility("default"))) int grng_probe_write_gbs(void* dev_buf,
                                                                             int64_t bytes,
                                                                             int reps,
                                                                             double* gbs) {
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return 4;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n16 = bytes / 16;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int grid = sms * 16;
  for (int i = 0; i < 2; ++i) probe_store<<<grid, 256>>>((uint4*)dev_buf, n16);
  cudaEventRecord(a);
  for (int i = 0; i < reps; ++i) probe_store<<<grid, 256>>>((uint4*)dev_buf, n16);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *gbs = (double)n16 * 16.0 * reps / (ms * 1e-3) / 1e9;
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

extern "C" __attribute__((visibility("default"))) int grng_probe_mulwide_rate(void* dev_sink,
                                                                                double* per_s) {
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return 4;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 8, iters = 4096;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int reps = 5;
  double best = 0.0;
  for (int shape = 0; shape < 2; ++shape) {
    // both shapes: 8 products per thread per iteration
    auto launch = [&](uint32_t seed) {
      if (shape == 0)
        probe_mulwide<<<grid, 256>>>((uint32_t*)dev_sink, iters, seed);
      else
        probe_mulwide_cross<<<grid, 256>>>((uint32_t*)dev_sink, iters, seed);
    };
    launch(1u);
    cudaEventRecord(a);
    for (int i = 0; i < reps; ++i) launch(2u + i);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double r = (double)grid * 256.0 * iters * 8.0 * reps / (ms * 1e-3);
    if (r > best) best = r;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *per_s = best;
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
