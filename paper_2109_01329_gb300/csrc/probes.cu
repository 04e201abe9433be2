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

}  // namespace

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
