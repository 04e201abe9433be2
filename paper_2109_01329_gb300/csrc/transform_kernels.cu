// Distribution transform of caller-supplied words (grng_transform_words):
// one thread per unit (one output, or one Box-Muller pair), the same
// unit_outputs<V> as the fused fill kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "grng_internal.h"

namespace grng {
namespace {

using namespace dev;

template <int V>
__global__ void __launch_bounds__(256) transform_kernel(TransformParams t, const uint32_t* words,
                                                        int64_t n, uint32_t* out) {
  using I = VInfo<V>;
  const int64_t units = (n + I::epu - 1) / I::epu;
  const int64_t out_words = n * I::ow_per_elem;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < units;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint32_t w[I::wpu];
#pragma unroll
    for (int i = 0; i < I::wpu; ++i) w[i] = words[k * I::wpu + i];
    uint32_t o[I::wpu];
    // odd units take the other pipe's form as in the fill kernels (the same
    // bits), so this kernel checks both forms
    unit_outputs<V>(w, o, t, (k & 1) != 0);
#pragma unroll
    for (int i = 0; i < I::wpu; ++i) {
      const int64_t ow = k * I::wpu + i;  // 4 output bytes per word
      if (ow < out_words) out[ow] = o[i];
    }
  }
}

template <int V>
grng_status launch_v(const TransformParams& t, const uint32_t* words, int64_t n, void* out,
                     cudaStream_t stream) {
  using I = VInfo<V>;
  const int64_t units = (n + I::epu - 1) / I::epu;
  int dev = 0;
  const int sms = current_device_sms(&dev);
  int64_t grid = (units + 255) / 256;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  transform_kernel<V><<<(unsigned)grid, 256, 0, stream>>>(t, words, n,
                                                          reinterpret_cast<uint32_t*>(out));
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error("transform launch failed: %s", cudaGetErrorString(err));
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}

}  // namespace

grng_status launch_transform(int variant, const TransformParams& t, const uint32_t* words,
                             int64_t n, void* out, CUstream_st* stream) {
  switch (variant) {
    case V_BITS: return launch_v<V_BITS>(t, words, n, out, stream);
    case V_U01_F32: return launch_v<V_U01_F32>(t, words, n, out, stream);
    case V_UNI_F32: return launch_v<V_UNI_F32>(t, words, n, out, stream);
    case V_U01_F64: return launch_v<V_U01_F64>(t, words, n, out, stream);
    case V_AFF_F64: return launch_v<V_AFF_F64>(t, words, n, out, stream);
    case V_UNI_F64: return launch_v<V_UNI_F64>(t, words, n, out, stream);
    case V_GAUSS_F32: return launch_v<V_GAUSS_F32>(t, words, n, out, stream);
    case V_LOGN_F32: return launch_v<V_LOGN_F32>(t, words, n, out, stream);
    case V_GAUSS_F64: return launch_v<V_GAUSS_F64>(t, words, n, out, stream);
    case V_LOGN_F64: return launch_v<V_LOGN_F64>(t, words, n, out, stream);
    case V_ICDF_GAUSS_F32: return launch_v<V_ICDF_GAUSS_F32>(t, words, n, out, stream);
    case V_ICDF_LOGN_F32: return launch_v<V_ICDF_LOGN_F32>(t, words, n, out, stream);
    case V_ICDF_GAUSS_F64: return launch_v<V_ICDF_GAUSS_F64>(t, words, n, out, stream);
    case V_ICDF_LOGN_F64: return launch_v<V_ICDF_LOGN_F64>(t, words, n, out, stream);
    case V_STDGAUSS_F64: return launch_v<V_STDGAUSS_F64>(t, words, n, out, stream);
    default: set_error("unknown variant %d", variant); return GRNG_ERR_INVALID_ARG;
  }
}

}  // namespace grng
