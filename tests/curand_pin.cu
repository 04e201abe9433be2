// Test infrastructure: cuRAND's device API (curand_kernel.h) driven as a black
// box, an implementation of Philox4x32-10 and MRG32k3a written independently
// of this repository.  The oracle's pins compare the oracle's engines with it
// (tests/test_gpu_curand_pin.py).  Nothing here is part of the library.
//
// Each entry point runs one CUDA thread that sets a generator state from the
// caller's words, draws k values in turn and copies them back to the host.
// The output buffer holds exactly k values and the loop writes indices
// 0 .. k - 1 only.
#include <cuda_runtime.h>
#include <curand_kernel.h>

namespace {

__global__ void mrg_uniforms_kernel(const unsigned* s, int k, double* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  curandStateMRG32k3a_t st;
  for (int i = 0; i < 3; ++i) {
    st.s1[i] = s[i];
    st.s2[i] = s[3 + i];
  }
  st.boxmuller_flag = 0;
  st.boxmuller_flag_double = 0;
  st.boxmuller_extra = 0.0f;
  st.boxmuller_extra_double = 0.0;
  for (int i = 0; i < k; ++i) out[i] = curand_uniform_double(&st);
}

__global__ void philox_blocks_kernel(uint4 ctr, uint2 key, int k, uint4* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  curandStatePhilox4_32_10_t st;
  st.ctr = ctr;
  st.key = key;
  st.output = make_uint4(0u, 0u, 0u, 0u);
  st.STATE = 0;
  st.boxmuller_flag = 0;
  st.boxmuller_flag_double = 0;
  st.boxmuller_extra = 0.0f;
  st.boxmuller_extra_double = 0.0;
  for (int i = 0; i < k; ++i) out[i] = curand4(&st);
}

constexpr int kMaxK = 1 << 16;

}  // namespace

// state[0..2] -> s1, state[3..5] -> s2; out receives k doubles.
// Returns 0, or a CUDA error code (k outside 1..65536: -1).
extern "C" int pin_mrg_uniforms(const unsigned* state, int k, double* out) {
  if (k < 1 || k > kMaxK) return -1;
  unsigned* d_s = nullptr;
  double* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_s, 6 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)k * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d_s, state, 6 * sizeof(unsigned), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    mrg_uniforms_kernel<<<1, 1>>>(d_s, k, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_s);
  cudaFree(d_out);
  return (int)e;
}

// ctr[0..3] = counter words, key[0..1] = key words; out receives 4 k words.
extern "C" int pin_philox_blocks(const unsigned* ctr, const unsigned* key, int k, unsigned* out) {
  if (k < 1 || k > kMaxK) return -1;
  uint4* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_out, (size_t)k * sizeof(uint4));
  if (e == cudaSuccess) {
    philox_blocks_kernel<<<1, 1>>>(make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]),
                                   make_uint2(key[0], key[1]), k, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, (size_t)k * sizeof(uint4), cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  return (int)e;
}
