// grng_generate_host_static: generate-to-host for callers that cannot
// allocate device memory.
//
// grng_generate_host needs a device staging buffer from its caller.  Some
// callers cannot provide one at the point of the call: a host application
// whose memory pool has already reserved the whole device, code where
// cudaMalloc / cudaFree are not allowed because they may synchronise the
// device (latency-critical threads, callbacks), or plug-ins whose host
// forbids device allocations after start-up.  This entry point stages through
// a fixed array that lives in the library's own module instead, so it makes
// no allocation of any kind.
//
// The array costs kStageBytes of device memory on every GPU that loads the
// library, held until the process exits.  It is shared by every call in the
// process; a mutex serialises the calls and each call waits for its copy
// before returning, so two calls never overlap on the GPU within one
// process.  Calls that did overlap on the GPU would race on the array.
// Nothing in the array has to start at zero: a call writes every element it
// copies out before copying it.  The array's device address is looked up
// once per device and kept; after cudaDeviceReset the module is loaded anew
// at another address, so the entry point must not be used on a device that
// was reset in the same process.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "grng.h"
#include "grng_internal.h"

namespace grng {
namespace {

constexpr size_t kStageBytes = GRNG_STATIC_STAGE_BYTES;
constexpr int kMaxDevices = 256;

__device__ __align__(256) unsigned char g_static_stage[kStageBytes];

std::mutex g_static_mutex;
void* g_stage_addr[kMaxDevices];  // device address of g_static_stage, per device

}  // namespace
}  // namespace grng

using namespace grng;

extern "C" grng_status grng_generate_host_static(const grng_distribution* dist,
                                                 grng_engine_t engine, int64_t n, void* host_ptr,
                                                 grng_stream_t stream) {
  uint64_t words = 0;
  grng_status st = grng_words_for(dist, n, &words);  // checks dist and n
  if (st != GRNG_OK) return st;
  if (engine == nullptr) {
    set_error("engine is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  const uint64_t es = dist->dtype == GRNG_F64 ? 8u : 4u;
  if ((uint64_t)n * es > (uint64_t)kStageBytes) {
    set_error("n * element size = %llu bytes exceeds the %llu-byte static staging array; "
              "split the request into several calls",
              (unsigned long long)((uint64_t)n * es), (unsigned long long)kStageBytes);
    return GRNG_ERR_UNSUPPORTED;
  }
  if (n == 0) return GRNG_OK;
  if (host_ptr == nullptr) {
    set_error("host_ptr is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mutex);
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) {
    set_error("cudaGetDevice failed: %s", cudaGetErrorString(err));
    cudaGetLastError();
    return GRNG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d is outside the %d devices this entry point supports", dev,
              kMaxDevices);
    return GRNG_ERR_UNSUPPORTED;
  }
  // Set-up, once per device, with that device current: the host-side name
  // g_static_stage is only a stand-in, the kernel needs the device address.
  if (g_stage_addr[dev] == nullptr) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_static_stage);
    if (err != cudaSuccess || p == nullptr) {
      set_error("cudaGetSymbolAddress of the static staging array failed: %s",
                cudaGetErrorString(err));
      cudaGetLastError();
      return GRNG_ERR_CUDA;
    }
    g_stage_addr[dev] = p;
  }
  void* stage = g_stage_addr[dev];
  st = grng_generate(dist, engine, n, stage, stream);  // advances the engine on success
  if (st != GRNG_OK) return st;
  err = cudaMemcpyAsync(host_ptr, stage, (size_t)n * es, cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    set_error("copying the staged output to the host failed: %s", cudaGetErrorString(err));
    cudaGetLastError();
    // put the engine back where it was: advancing by 2^128 - words wraps to -words
    const uint64_t back_lo = ~words + 1u;
    const uint64_t back_hi = words == 0 ? 0u : ~uint64_t(0);
    grng_engine_skip_ahead(engine, back_lo, back_hi);
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}
