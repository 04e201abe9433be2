// Launch-geometry table of the single-stream fills and its autotuner.
//
// The paper's future work (Sec. 8) expects kernels written for the hardware
// to need tuning; Sec. 7 shows the launch configuration mattering (the
// transform kernel ran at 1024 threads per block where the native library
// chose 256).  Every fill's output is a function of its word index only, so
// the geometry changes speed, never values.  The geometry of a fill is one
// integer per (engine, kernel variant, size bucket), the bucket being the bit
// length of n:
//   Philox4x32-10: the CTAs per SM of the grid, the kernels looping with a
//     grid stride: 1..16 caps the resident CTAs (fewer CTAs give each thread
//     more blocks), 17 and above launches (value - 16) waves of resident CTAs;
//   MRG32k3a: the threads per SM of the chunk plan in units of 256 (the
//     chunk length, hence the jump-ahead work per output, follows from it).
// 0 keeps the launcher's built-in choice (Philox: 8 waves of resident CTAs;
// MRG32k3a: 2048 threads per SM).  The table starts from the file named by
// the environment variable GRNG_TUNE_CACHE, if set, when it is first read;
// grng_fill_autotune fills entries by timing, grng_tune_save / _load write and
// read the text format "grng-tune 1" followed by lines
// "engine variant bucket geometry".
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "grng.h"
#include "grng_internal.h"

namespace grng {
namespace {

constexpr int kBuckets = 64;
std::atomic<int32_t> g_geom[2][V_COUNT][kBuckets];
std::once_flag g_env_once;

int bucket_of(int64_t n) {
  int b = 0;
  while (n > 0 && b < kBuckets - 1) {
    ++b;
    n >>= 1;
  }
  return b;
}

grng_status load_file(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) {
    set_error("cannot open tune file %s", path);
    return GRNG_ERR_INVALID_ARG;
  }
  char head[32] = {0};
  int ver = 0;
  if (std::fscanf(f, "%31s %d", head, &ver) != 2 || std::strcmp(head, "grng-tune") != 0 ||
      ver != 1) {
    std::fclose(f);
    set_error("%s is not a grng-tune 1 file", path);
    return GRNG_ERR_INVALID_ARG;
  }
  int e = 0, v = 0, b = 0, g = 0;
  grng_status st = GRNG_OK;
  while (true) {
    const int k = std::fscanf(f, "%d %d %d %d", &e, &v, &b, &g);
    if (k == EOF) break;
    if (k != 4 || e < 0 || e > 1 || v < 0 || v >= V_COUNT || b < 0 || b >= kBuckets || g < 0 ||
        g > 64) {
      set_error("bad entry in tune file %s", path);
      st = GRNG_ERR_INVALID_ARG;
      break;
    }
    g_geom[e][v][b].store(g, std::memory_order_relaxed);
  }
  std::fclose(f);
  return st;
}

void load_env() {
  const char* p = std::getenv("GRNG_TUNE_CACHE");
  if (p != nullptr && p[0] != '\0') {
    FILE* f = std::fopen(p, "r");
    if (f != nullptr) {  // a cache that does not exist yet is not an error
      std::fclose(f);
      load_file(p);
    }
  }
}

}  // namespace

int32_t fill_geometry(int engine_kind, int variant, int64_t n) {
  std::call_once(g_env_once, load_env);
  if (engine_kind < 0 || engine_kind > 1 || variant < 0 || variant >= V_COUNT) return 0;
  return g_geom[engine_kind][variant][bucket_of(n)].load(std::memory_order_relaxed);
}

}  // namespace grng

using namespace grng;

extern "C" {

grng_status grng_fill_set_geometry(int32_t engine_kind, const grng_distribution* dist, int64_t n,
                                   int32_t geometry) {
  TransformParams t;
  int v = 0;
  grng_status st = fill_transform_params(dist, &t, &v);
  if (st != GRNG_OK) return st;
  if ((engine_kind != GRNG_PHILOX4X32X10 && engine_kind != GRNG_MRG32K3A) || n < 0 ||
      geometry < 0 || geometry > 64) {
    set_error("bad engine kind, n < 0 or geometry outside 0..64");
    return GRNG_ERR_INVALID_ARG;
  }
  std::call_once(g_env_once, load_env);
  g_geom[engine_kind][v][bucket_of(n)].store(geometry, std::memory_order_relaxed);
  return GRNG_OK;
}

grng_status grng_fill_get_geometry(int32_t engine_kind, const grng_distribution* dist, int64_t n,
                                   int32_t* geometry) {
  TransformParams t;
  int v = 0;
  grng_status st = fill_transform_params(dist, &t, &v);
  if (st != GRNG_OK) return st;
  if ((engine_kind != GRNG_PHILOX4X32X10 && engine_kind != GRNG_MRG32K3A) || n < 0 ||
      geometry == nullptr) {
    set_error("bad engine kind, n < 0 or geometry NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  *geometry = fill_geometry(engine_kind, v, n);
  return GRNG_OK;
}

grng_status grng_fill_autotune(int32_t engine_kind, const grng_distribution* dist, int64_t n,
                               void* dev_buf, grng_stream_t stream_in, int32_t* best_geometry,
                               float* best_ms, float* builtin_ms) {
  TransformParams t;
  int v = 0;
  grng_status st = fill_transform_params(dist, &t, &v);
  if (st != GRNG_OK) return st;
  if ((engine_kind != GRNG_PHILOX4X32X10 && engine_kind != GRNG_MRG32K3A) || n < 1 ||
      dev_buf == nullptr) {
    set_error("bad engine kind, n < 1 or dev_buf NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  cudaStream_t stream = (cudaStream_t)stream_in;
  grng_engine_t e = nullptr;
  st = grng_engine_create(&e, engine_kind, 0x5EEDu, 0);
  if (st != GRNG_OK) return st;
  static const int32_t kPhilox[] = {0, 1, 2, 4, 17, 18, 20, 32, 48, 64};
  static const int32_t kMrg[] = {0, 1, 2, 4, 6, 12, 16};
  const int32_t* cand = engine_kind == GRNG_PHILOX4X32X10 ? kPhilox : kMrg;
  const int ncand = engine_kind == GRNG_PHILOX4X32X10 ? 10 : 7;
  std::call_once(g_env_once, load_env);
  std::atomic<int32_t>& slot = g_geom[engine_kind][v][bucket_of(n)];
  const int32_t before = slot.load(std::memory_order_relaxed);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("event creation failed");
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    grng_engine_destroy(e);
    return GRNG_ERR_CUDA;
  }
  float best = 1e30f, t_builtin = 0.f;
  int32_t arg = before;
  for (int i = 0; i < ncand && st == GRNG_OK; ++i) {
    slot.store(cand[i], std::memory_order_relaxed);
    st = grng_generate(dist, e, n, dev_buf, stream_in);  // warm-up
    if (st != GRNG_OK) break;
    cudaEventRecord(e0, stream);
    for (int k = 0; k < 3 && st == GRNG_OK; ++k) st = grng_generate(dist, e, n, dev_buf, stream_in);
    cudaEventRecord(e1, stream);
    if (st != GRNG_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("fill autotune: timing failed");
      cudaGetLastError();
      st = GRNG_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cand[i] == 0) t_builtin = ms / 3;
    if (ms / 3 < best * 0.99f) {  // ties keep the earlier (the built-in choice first)
      best = ms / 3;
      arg = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  grng_engine_destroy(e);
  slot.store(st == GRNG_OK ? arg : before, std::memory_order_relaxed);
  if (st != GRNG_OK) return st;
  if (best_geometry) *best_geometry = arg;
  if (best_ms) *best_ms = best;
  if (builtin_ms) *builtin_ms = t_builtin;
  return GRNG_OK;
}

grng_status grng_tune_save(const char* path) {
  if (path == nullptr) {
    set_error("path is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::call_once(g_env_once, load_env);
  FILE* f = std::fopen(path, "w");
  if (f == nullptr) {
    set_error("cannot write tune file %s", path);
    return GRNG_ERR_INVALID_ARG;
  }
  std::fprintf(f, "grng-tune 1\n");
  for (int e = 0; e < 2; ++e)
    for (int v = 0; v < V_COUNT; ++v)
      for (int b = 0; b < kBuckets; ++b) {
        const int32_t g = g_geom[e][v][b].load(std::memory_order_relaxed);
        if (g != 0) std::fprintf(f, "%d %d %d %d\n", e, v, b, g);
      }
  const bool ok = std::fclose(f) == 0;
  if (!ok) {
    set_error("writing tune file %s failed", path);
    return GRNG_ERR_INVALID_ARG;
  }
  return GRNG_OK;
}

grng_status grng_tune_load(const char* path) {
  if (path == nullptr) {
    set_error("path is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::call_once(g_env_once, load_env);
  return load_file(path);
}

grng_status grng_tune_reset(void) {
  std::call_once(g_env_once, load_env);
  for (int e = 0; e < 2; ++e)
    for (int v = 0; v < V_COUNT; ++v)
      for (int b = 0; b < kBuckets; ++b) g_geom[e][v][b].store(0, std::memory_order_relaxed);
  return GRNG_OK;
}

}  // extern "C"
