// Batched generation: many independent Philox requests in one persistent
// launch (the event batching the paper leaves as future work, Sec. 7, and the
// small-batch latency it measures, Sec. 7 / Fig. 2-4).
//
// A batch is planned once on the host (grng_batch_create): per request its
// variant, parameters, output pointer, 16-byte group count and starting word
// offset; a tile -> request map; and per request the words its engine
// advances per launch.  The tables live in a caller-provided device
// workspace.  grng_batch_launch then enqueues two kernels:
//   1. batch_fill_kernel: CTAs walk the tiles (a tile is kThreads * ipt
//      16-byte groups of one request) with a static grid stride; each thread
//      produces ipt groups of its tile;
//   2. batch_advance_kernel: adds each request's advance to its device-
//      resident 128-bit offset,
// so launching again (or replaying a CUDA graph of the launch) continues every
// generator's sequence with no host work.  grng_batch_commit copies the device
// offsets back into the engines.
//
// A request whose word offset matches its pointer's 16-byte phase maps each
// 16-byte group to one Philox block; at any other phase a warp computes 32
// consecutive blocks and exchanges the straddling words by shuffle (no
// shared memory anywhere).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "device_common.cuh"
#include "grng.h"
#include "grng_internal.h"

namespace grng {

namespace {

using namespace dev;

constexpr int kThreads = 256;

// Workspace layout (each part 256-byte aligned):
//   BatchReq reqs[count] | uint64_t off[count][2] | int32_t tile_req[tiles]
size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

// Stores the elements of group (first element e0) that lie in [0, n).
template <int V>
__device__ __forceinline__ void store_group(char* base, int64_t e0, int64_t n, uint4 o) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  if (e0 >= 0 && e0 + kEpg <= n) {
    store16(base + e0 * I::es, o);
    return;
  }
  const uint32_t ow[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
  for (int i = 0; i < kEpg; ++i) {
    const int64_t e = e0 + i;
    if (e >= 0 && e < n) {
      if constexpr (I::es == 4) {
        reinterpret_cast<uint32_t*>(base)[e] = ow[i];
      } else {
        reinterpret_cast<uint2*>(base)[e] = make_uint2(ow[2 * i], ow[2 * i + 1]);
      }
    }
  }
}

// The groups [g0, g0 + kThreads ipt) of one request (the whole CTA works on
// one tile, so every branch below is uniform across it).  Group 0 starts
// head elements (pw = head es / 4 words) before the output.  When pw is a
// multiple of the unit size, group g is the 4 words from word off - pw + 4 g:
// exactly Philox block (off - pw)/4 + g when off - pw is a multiple of 4,
// else the tail of one block and the head of the next, exchanged between
// neighbouring lanes.  Otherwise (a Box-Muller pair split by the output's
// start) lanes transform pair-aligned virtual groups one element earlier and
// exchange the straddling element by shuffle.
template <int V>
__device__ __forceinline__ void batch_tile(const BatchReq& r, uint64_t off_lo, uint64_t off_hi,
                                           int64_t g0, int ipt) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  constexpr int kWpu = I::wpu, kEpu = I::epu;
  const int64_t n = r.n, groups = r.groups, head = r.head;
  const uint32_t k0 = r.key0, k1 = r.key1;
  char* base = reinterpret_cast<char*>(r.out);
  const TransformParams t = r.t;
  const uint32_t pw = (uint32_t)head * (uint32_t)(I::es / 4);
  if ((pw % (uint32_t)kWpu) == 0) {
    // group g is the 4 words from word off - pw + 4 g: the block of that
    // word from phase ph on, and the first ph words of the next block
    const uint64_t a_lo = off_lo - pw, a_hi = off_hi - ((off_lo < pw) ? 1u : 0u);
    const uint64_t b_lo = (a_lo >> 2) | (a_hi << 62), b_hi = a_hi >> 2;
    const uint32_t ph = (uint32_t)a_lo & 3u;
    if (ph == 0) {
      for (int i = 0; i < ipt; ++i) {
        const int64_t g = g0 + (int64_t)i * kThreads + threadIdx.x;
        if (g >= groups) break;
        const uint64_t c_lo = b_lo + (uint64_t)g;
        const uint64_t c_hi = b_hi + ((c_lo < b_lo) ? 1u : 0u);
        const uint4 o = block_outputs<V>(philox4x32_10(ctr_from(c_lo, c_hi), k0, k1), t);
        store_group<V>(base, g * kEpg - head, n, o);
      }
      return;
    }
    // Each warp computes 32 consecutive blocks and emits the 31 groups that
    // start in its lanes 0..30, taking the next block's words from lane + 1
    // by shuffle: no shared memory and no barrier.  The loop bound depends
    // only on the warp, so every shuffle has all 32 lanes.
    const int lane = threadIdx.x & 31;
    const int64_t g_end = (g0 + (int64_t)kThreads * ipt) < groups ? (g0 + (int64_t)kThreads * ipt)
                                                                   : groups;
    constexpr int kPerWarp = 31;
    for (int64_t gs = g0 + (int64_t)(threadIdx.x >> 5) * kPerWarp; gs < g_end;
         gs += (int64_t)kPerWarp * (kThreads / 32)) {
      const int64_t g = gs + lane;
      const uint64_t c_lo = b_lo + (uint64_t)g;
      const uint64_t c_hi = b_hi + ((c_lo < b_lo) ? 1u : 0u);
      const uint4 b = philox4x32_10(ctr_from(c_lo, c_hi), k0, k1);
      const uint32_t n0 = __shfl_down_sync(0xFFFFFFFFu, b.x, 1);
      const uint32_t n1 = __shfl_down_sync(0xFFFFFFFFu, b.y, 1);
      const uint32_t n2 = __shfl_down_sync(0xFFFFFFFFu, b.z, 1);
      uint4 w;
      if (ph == 1) {
        w = make_uint4(b.y, b.z, b.w, n0);
      } else if (ph == 2) {
        w = make_uint4(b.z, b.w, n0, n1);
      } else {
        w = make_uint4(b.w, n0, n1, n2);
      }
      if (lane < kPerWarp && g < g_end) store_group<V>(base, g * kEpg - head, n, block_outputs<V>(w, t));
    }
    return;
  }
  if constexpr (kEpu == 2) {
    // A Box-Muller pair split by the output's start (odd head): virtual group
    // g starts one element before output group g, on a pair boundary, at
    // word off - pw - es / 4 + 4 g.  Each lane transforms its virtual group
    // (words from its block and, at a non-zero phase, the next lane's) and
    // output group g is virtual group g without its first element plus the
    // first element of virtual group g + 1, taken from lane + 1: 30 groups
    // per warp, every pair transformed once, no shared memory.
    constexpr uint32_t kPv = (uint32_t)(I::es / 4);
    const uint64_t a_lo = off_lo - (pw + kPv);
    const uint64_t a_hi = off_hi - ((off_lo < (uint64_t)(pw + kPv)) ? 1u : 0u);
    const uint64_t b_lo = (a_lo >> 2) | (a_hi << 62), b_hi = a_hi >> 2;
    const uint32_t ph = (uint32_t)a_lo & 3u;
    const int lane = threadIdx.x & 31;
    const int64_t g_end = (g0 + (int64_t)kThreads * ipt) < groups ? (g0 + (int64_t)kThreads * ipt)
                                                                   : groups;
    constexpr int kPerWarp = 30;
    for (int64_t gs = g0 + (int64_t)(threadIdx.x >> 5) * kPerWarp; gs < g_end;
         gs += (int64_t)kPerWarp * (kThreads / 32)) {
      const int64_t g = gs + lane;
      const uint64_t c_lo = b_lo + (uint64_t)g;
      const uint64_t c_hi = b_hi + ((c_lo < b_lo) ? 1u : 0u);
      const uint4 b = philox4x32_10(ctr_from(c_lo, c_hi), k0, k1);
      const uint32_t n0 = __shfl_down_sync(0xFFFFFFFFu, b.x, 1);
      const uint32_t n1 = __shfl_down_sync(0xFFFFFFFFu, b.y, 1);
      const uint32_t n2 = __shfl_down_sync(0xFFFFFFFFu, b.z, 1);
      uint4 w = b;
      if (ph == 1) {
        w = make_uint4(b.y, b.z, b.w, n0);
      } else if (ph == 2) {
        w = make_uint4(b.z, b.w, n0, n1);
      } else if (ph == 3) {
        w = make_uint4(b.w, n0, n1, n2);
      }
      const uint4 v = block_outputs<V>(w, t);
      const uint32_t m0 = __shfl_down_sync(0xFFFFFFFFu, v.x, 1);
      const uint32_t m1 = __shfl_down_sync(0xFFFFFFFFu, v.y, 1);
      const uint4 o = I::es == 4 ? make_uint4(v.y, v.z, v.w, m0) : make_uint4(v.z, v.w, m0, m1);
      if (lane < kPerWarp && g < g_end) store_group<V>(base, g * kEpg - head, n, o);
    }
  }
}

__global__ void __launch_bounds__(kThreads) batch_fill_kernel(const BatchReq* __restrict__ reqs,
                                                              const uint64_t* __restrict__ off,
                                                              const int32_t* __restrict__ tile_req,
                                                              int64_t tiles, int ipt) {
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int32_t ri = tile_req[t];
    const BatchReq& r = reqs[ri];
    const uint64_t off_lo = off[2 * ri], off_hi = off[2 * ri + 1];
    const int64_t g0 = (t - r.first_tile) * (int64_t)kThreads * ipt;
    switch (r.variant) {  // uniform per tile
      case V_BITS: batch_tile<V_BITS>(r, off_lo, off_hi, g0, ipt); break;
      case V_U01_F32: batch_tile<V_U01_F32>(r, off_lo, off_hi, g0, ipt); break;
      case V_UNI_F32: batch_tile<V_UNI_F32>(r, off_lo, off_hi, g0, ipt); break;
      case V_U01_F64: batch_tile<V_U01_F64>(r, off_lo, off_hi, g0, ipt); break;
      case V_AFF_F64: batch_tile<V_AFF_F64>(r, off_lo, off_hi, g0, ipt); break;
      case V_UNI_F64: batch_tile<V_UNI_F64>(r, off_lo, off_hi, g0, ipt); break;
      case V_GAUSS_F32: batch_tile<V_GAUSS_F32>(r, off_lo, off_hi, g0, ipt); break;
      case V_LOGN_F32: batch_tile<V_LOGN_F32>(r, off_lo, off_hi, g0, ipt); break;
      case V_GAUSS_F64: batch_tile<V_GAUSS_F64>(r, off_lo, off_hi, g0, ipt); break;
      case V_LOGN_F64: batch_tile<V_LOGN_F64>(r, off_lo, off_hi, g0, ipt); break;
      case V_ICDF_GAUSS_F32: batch_tile<V_ICDF_GAUSS_F32>(r, off_lo, off_hi, g0, ipt); break;
      case V_ICDF_LOGN_F32: batch_tile<V_ICDF_LOGN_F32>(r, off_lo, off_hi, g0, ipt); break;
      case V_ICDF_GAUSS_F64: batch_tile<V_ICDF_GAUSS_F64>(r, off_lo, off_hi, g0, ipt); break;
      case V_STDGAUSS_F64: batch_tile<V_STDGAUSS_F64>(r, off_lo, off_hi, g0, ipt); break;
      default: batch_tile<V_ICDF_LOGN_F64>(r, off_lo, off_hi, g0, ipt); break;
    }
  }
}

__global__ void batch_advance_kernel(const BatchReq* __restrict__ reqs, uint64_t* off,
                                     int32_t count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint64_t lo = off[2 * i] + reqs[i].adv_lo;
  off[2 * i + 1] += reqs[i].adv_hi + ((lo < off[2 * i]) ? 1u : 0u);
  off[2 * i] = lo;
}

}  // namespace

int64_t plan_parts(const PartDesc* parts, int32_t count, int ipt, BatchReq* reqs_out,
                   uint64_t* offs_out, int32_t* tiles_out, int64_t tile_cap) {
  const int64_t tile_groups = (int64_t)kThreads * ipt;
  int64_t t = 0;
  for (int32_t i = 0; i < count; ++i) {
    const PartDesc& q = parts[i];
    BatchReq& r = reqs_out[i];
    std::memset(&r, 0, sizeof(r));
    const int64_t epg = 16 / q.es;
    const int32_t head = (int32_t)((q.out & 15u) / (uint64_t)q.es);
    const int64_t groups = q.n == 0 ? 0 : (head + q.n + epg - 1) / epg;
    r.t = q.t;
    r.out = q.out;
    r.n = q.n;
    r.groups = groups;
    r.first_tile = t;
    r.variant = q.variant;
    r.head = head;
    r.key0 = q.key0;
    r.key1 = q.key1;
    offs_out[2 * i] = q.off_lo;
    offs_out[2 * i + 1] = q.off_hi;
    const int64_t nt = (groups + tile_groups - 1) / tile_groups;
    if (t + nt > tile_cap) return -1;
    for (int64_t k = 0; k < nt; ++k) tiles_out[t + k] = i;
    t += nt;
  }
  return t;
}

grng_status enqueue_fill(const BatchReq* d_reqs, const uint64_t* d_offs, const int32_t* d_tiles,
                         int64_t tiles, int ipt, int64_t grid, cudaStream_t stream) {
  if (tiles <= 0) return GRNG_OK;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  batch_fill_kernel<<<(unsigned)grid, kThreads, 0, stream>>>(d_reqs, d_offs, d_tiles, tiles, ipt);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error("batch fill launch failed: %s", cudaGetErrorString(err));
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}

}  // namespace grng

struct grng_batch {
  int32_t count;
  int64_t tiles;
  int32_t ipt;           // groups per thread per tile
  int32_t ctas_per_sm;
  int32_t sms;
  int32_t device;
  void* workspace;
  size_t workspace_bytes;
  size_t reqs_off, offs_off, tiles_off;
  std::vector<grng::BatchReq> host_reqs;  // the request records as uploaded
  std::vector<int64_t> groups;            // per request
  int64_t groups_total;
  std::vector<grng_engine_t> engines;  // per request
  std::vector<int32_t> first_req_of_engine;  // per request: index of its engine's first request
  std::vector<uint64_t> start_lo, start_hi;  // per request: start offset at creation
};

using namespace grng;

namespace {

constexpr int32_t kMaxBatch = 1 << 20;

grng_status plan_sizes(const grng_request* reqs, int32_t count, int ipt, int64_t* tiles_out,
                       std::vector<int64_t>* groups, std::vector<int32_t>* heads,
                       std::vector<int>* variants, std::vector<TransformParams>* tps) {
  int64_t tiles = 0;
  const int64_t tile_groups = (int64_t)kThreads * ipt;
  for (int32_t i = 0; i < count; ++i) {
    const grng_request& q = reqs[i];
    uint64_t words = 0;
    grng_status st = grng_words_for(&q.dist, q.n, &words);
    if (st != GRNG_OK) return st;
    if (q.engine == nullptr) {
      set_error("request %d: engine is NULL", i);
      return GRNG_ERR_INVALID_ARG;
    }
    grng_engine_state es;
    grng_engine_get_state(q.engine, &es);
    if (es.kind != GRNG_PHILOX4X32X10) {
      set_error("request %d: batches take Philox4x32-10 engines", i);
      return GRNG_ERR_UNSUPPORTED;
    }
    const int esz = q.dist.dtype == GRNG_F64 ? 8 : 4;
    if ((q.n > 0 && q.out == nullptr) || ((uintptr_t)q.out % (uintptr_t)esz) != 0) {
      set_error("request %d: output pointer NULL or misaligned", i);
      return GRNG_ERR_INVALID_ARG;
    }
    TransformParams t;
    int v = 0;
    st = fill_transform_params(&q.dist, &t, &v);
    if (st != GRNG_OK) return st;
    const int32_t head = (int32_t)(((uintptr_t)q.out & 15u) / (uintptr_t)esz);
    const int64_t epg = 16 / esz;
    const int64_t g = q.n == 0 ? 0 : (head + q.n + epg - 1) / epg;
    groups->push_back(g);
    heads->push_back(head);
    variants->push_back(v);
    tps->push_back(t);
    tiles += (g + tile_groups - 1) / tile_groups;
  }
  *tiles_out = tiles;
  return GRNG_OK;
}

}  // namespace

extern "C" {

grng_status grng_batch_workspace_bytes(const grng_request* reqs, int32_t count, int32_t ipt,
                                       size_t* bytes) {
  if (reqs == nullptr || bytes == nullptr || count < 1 || count > kMaxBatch || ipt < 1 ||
      ipt > 64) {
    set_error("bad batch arguments (count in [1, 2^20], ipt in [1, 64])");
    return GRNG_ERR_INVALID_ARG;
  }
  std::vector<int64_t> groups;
  std::vector<int32_t> heads;
  std::vector<int> variants;
  std::vector<TransformParams> tps;
  int64_t tiles = 0;
  grng_status st = plan_sizes(reqs, count, ipt, &tiles, &groups, &heads, &variants, &tps);
  if (st != GRNG_OK) return st;
  *bytes = align256(sizeof(BatchReq) * (size_t)count) + align256(16u * (size_t)count) +
           align256(4u * (size_t)(tiles > 0 ? tiles : 1));
  return GRNG_OK;
}

grng_status grng_batch_create(grng_batch_t* out, const grng_request* reqs, int32_t count,
                              int32_t ipt, void* dev_workspace, size_t workspace_bytes,
                              grng_stream_t stream) {
  if (out == nullptr || dev_workspace == nullptr || ((uintptr_t)dev_workspace & 255u) != 0) {
    set_error("out NULL or workspace NULL / not 256-byte aligned");
    return GRNG_ERR_INVALID_ARG;
  }
  size_t need = 0;
  grng_status st = grng_batch_workspace_bytes(reqs, count, ipt, &need);
  if (st != GRNG_OK) return st;
  if (workspace_bytes < need) {
    set_error("workspace of %zu bytes is smaller than the %zu bytes needed", workspace_bytes, need);
    return GRNG_ERR_INVALID_ARG;
  }
  std::vector<int64_t> groups;
  std::vector<int32_t> heads;
  std::vector<int> variants;
  std::vector<TransformParams> tps;
  int64_t tiles = 0;
  st = plan_sizes(reqs, count, ipt, &tiles, &groups, &heads, &variants, &tps);
  if (st != GRNG_OK) return st;

  grng_batch* b = new (std::nothrow) grng_batch;
  if (b == nullptr) {
    set_error("batch allocation failed");
    return GRNG_ERR_OOM;
  }
  b->count = count;
  b->tiles = tiles;
  b->ipt = ipt;
  b->ctas_per_sm = 4;
  b->sms = current_device_sms(&b->device);
  b->workspace = dev_workspace;
  b->reqs_off = 0;
  b->offs_off = align256(sizeof(BatchReq) * (size_t)count);
  b->tiles_off = b->offs_off + align256(16u * (size_t)count);
  b->groups_total = 0;

  // Requests of one engine follow each other in its sequence, in table order.
  std::vector<BatchReq> h(count);
  std::vector<uint64_t> offs(2 * (size_t)count);
  std::vector<int32_t> tile_req((size_t)(tiles > 0 ? tiles : 1), 0);
  b->engines.resize(count);
  b->first_req_of_engine.resize(count);
  b->start_lo.resize(count);
  b->start_hi.resize(count);
  struct Acc {
    grng_engine_t e;
    uint64_t lo, hi;   // running offset
    int32_t first;
  };
  std::vector<Acc> acc;
  std::vector<int32_t> acc_of(count);
  std::unordered_map<grng_engine_t, int32_t> index_of;
  index_of.reserve((size_t)count * 2);
  for (int32_t i = 0; i < count; ++i) {
    int32_t a = -1;
    auto it = index_of.find(reqs[i].engine);
    if (it != index_of.end()) {
      a = it->second;
    } else {
      grng_engine_state es;
      grng_engine_get_state(reqs[i].engine, &es);
      acc.push_back({reqs[i].engine, es.offset_lo, es.offset_hi, i});
      a = (int32_t)acc.size() - 1;
      index_of.emplace(reqs[i].engine, a);
    }
    acc_of[i] = a;
    offs[2 * i] = acc[a].lo;
    offs[2 * i + 1] = acc[a].hi;
    b->start_lo[i] = acc[a].lo;
    b->start_hi[i] = acc[a].hi;
    uint64_t words = 0;
    grng_words_for(&reqs[i].dist, reqs[i].n, &words);
    const uint64_t lo = acc[a].lo + words;
    acc[a].hi += (lo < acc[a].lo) ? 1u : 0u;
    acc[a].lo = lo;
    b->engines[i] = reqs[i].engine;
    b->first_req_of_engine[i] = acc[a].first;
  }
  int64_t t = 0;
  const int64_t tile_groups = (int64_t)kThreads * ipt;
  for (int32_t i = 0; i < count; ++i) {
    BatchReq& r = h[i];
    std::memset(&r, 0, sizeof(r));
    r.t = tps[i];
    r.out = (uint64_t)(uintptr_t)reqs[i].out;
    r.n = reqs[i].n;
    r.groups = groups[i];
    r.first_tile = t;
    r.variant = variants[i];
    r.head = heads[i];
    grng_engine_state es;
    grng_engine_get_state(reqs[i].engine, &es);
    r.key0 = (uint32_t)es.seed;
    r.key1 = (uint32_t)(es.seed >> 32);
    // per launch the engine advances by all of its requests' words
    const Acc& A = acc[acc_of[i]];
    const uint64_t s_lo = b->start_lo[A.first], s_hi = b->start_hi[A.first];
    r.adv_lo = A.lo - s_lo;
    r.adv_hi = A.hi - s_hi - ((A.lo < s_lo) ? 1u : 0u);
    const int64_t nt = (groups[i] + tile_groups - 1) / tile_groups;
    for (int64_t k = 0; k < nt; ++k) tile_req[(size_t)(t + k)] = i;
    t += nt;
    b->groups_total += groups[i];
  }
  b->workspace_bytes = workspace_bytes;
  b->groups = groups;
  char* ws = reinterpret_cast<char*>(dev_workspace);
  cudaError_t err =
      cudaMemcpyAsync(ws + b->reqs_off, h.data(), sizeof(BatchReq) * (size_t)count,
                      cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(ws + b->offs_off, offs.data(), 16u * (size_t)count,
                          cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (err == cudaSuccess && tiles > 0)
    err = cudaMemcpyAsync(ws + b->tiles_off, tile_req.data(), 4u * (size_t)tiles,
                          cudaMemcpyHostToDevice, (cudaStream_t)stream);
  // the host vectors die here: wait for the copies
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    set_error("batch upload failed: %s", cudaGetErrorString(err));
    cudaGetLastError();
    delete b;
    return GRNG_ERR_CUDA;
  }
  b->host_reqs = std::move(h);
  *out = b;
  return GRNG_OK;
}

}  // extern "C"

namespace {

// Tiles of the batch at ipt groups per thread, and whether their map fits the
// workspace given at creation.
int64_t tiles_at(const grng_batch* b, int ipt) {
  const int64_t tile_groups = (int64_t)kThreads * ipt;
  int64_t t = 0;
  for (int64_t g : b->groups) t += (g + tile_groups - 1) / tile_groups;
  return t;
}
bool fits(const grng_batch* b, int ipt) {
  const int64_t t = tiles_at(b, ipt);
  return b->tiles_off + 4u * (size_t)(t > 0 ? t : 1) <= b->workspace_bytes;
}

// Rebuilds the tile map and the requests' first tiles for ipt and uploads
// both (synchronises the stream: the host tables are temporaries).
grng_status replan(grng_batch* b, int ipt, cudaStream_t stream) {
  if (ipt == b->ipt) return GRNG_OK;
  const int64_t tile_groups = (int64_t)kThreads * ipt;
  const int64_t tiles = tiles_at(b, ipt);
  std::vector<int32_t> tile_req((size_t)(tiles > 0 ? tiles : 1), 0);
  std::vector<BatchReq> h = b->host_reqs;
  int64_t t = 0;
  for (int32_t i = 0; i < b->count; ++i) {
    h[i].first_tile = t;
    const int64_t nt = (b->groups[i] + tile_groups - 1) / tile_groups;
    for (int64_t k = 0; k < nt; ++k) tile_req[(size_t)(t + k)] = i;
    t += nt;
  }
  // the offsets are not touched: the device copy is the live one
  char* ws = reinterpret_cast<char*>(b->workspace);
  cudaError_t err = cudaMemcpyAsync(ws + b->reqs_off, h.data(), sizeof(BatchReq) * h.size(),
                                    cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess && tiles > 0)
    err = cudaMemcpyAsync(ws + b->tiles_off, tile_req.data(), 4u * (size_t)tiles,
                          cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  if (err != cudaSuccess) {
    set_error("batch re-plan upload failed: %s", cudaGetErrorString(err));
    cudaGetLastError();
    return GRNG_ERR_CUDA;
  }
  b->host_reqs = std::move(h);
  b->ipt = ipt;
  b->tiles = tiles;
  return GRNG_OK;
}

}  // namespace

extern "C" {

grng_status grng_batch_set_config(grng_batch_t b, int32_t ipt, int32_t ctas_per_sm,
                                  grng_stream_t stream) {
  if (b == nullptr || ctas_per_sm < 1 || ctas_per_sm > 32 || ipt < 1 || ipt > 64) {
    set_error("bad batch, ipt (1..64) or ctas_per_sm (1..32)");
    return GRNG_ERR_INVALID_ARG;
  }
  if (!fits(b, ipt)) {
    set_error("the tile map at %d groups per thread does not fit the batch's workspace", ipt);
    return GRNG_ERR_INVALID_ARG;
  }
  const grng_status st = replan(b, ipt, (cudaStream_t)stream);
  if (st != GRNG_OK) return st;
  b->ctas_per_sm = ctas_per_sm;
  return GRNG_OK;
}

static grng_status batch_enqueue(grng_batch_t b, cudaStream_t stream, bool advance) {
  char* ws = reinterpret_cast<char*>(b->workspace);
  const BatchReq* reqs = reinterpret_cast<const BatchReq*>(ws + b->reqs_off);
  uint64_t* offs = reinterpret_cast<uint64_t*>(ws + b->offs_off);
  const int32_t* tile_req = reinterpret_cast<const int32_t*>(ws + b->tiles_off);
  if (b->tiles > 0) {
    int64_t grid = (int64_t)b->sms * b->ctas_per_sm;
    if (grid > b->tiles) grid = b->tiles;
    batch_fill_kernel<<<(unsigned)grid, kThreads, 0, stream>>>(reqs, offs, tile_req, b->tiles,
                                                               b->ipt);
  }
  if (advance)
    batch_advance_kernel<<<(b->count + 255) / 256, 256, 0, stream>>>(reqs, offs, b->count);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error("batch launch failed: %s", cudaGetErrorString(err));
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}

grng_status grng_batch_launch(grng_batch_t b, grng_stream_t stream) {
  if (b == nullptr) {
    set_error("batch is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  return batch_enqueue(b, (cudaStream_t)stream, true);
}

grng_status grng_batch_autotune(grng_batch_t b, grng_stream_t stream_in, int32_t* best_ipt,
                                int32_t* best_ctas, float* best_ms) {
  if (b == nullptr) {
    set_error("batch is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  cudaStream_t stream = (cudaStream_t)stream_in;
  const int32_t ipts[] = {1, 2, 4, 8, 16, 32};
  const int32_t ctas[] = {1, 2, 4, 6, 8, 12, 16};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("event creation failed");
    cudaGetLastError();
    return GRNG_ERR_CUDA;
  }
  float best = 1e30f;
  int32_t arg_ipt = b->ipt, arg_ctas = b->ctas_per_sm;
  grng_status st = GRNG_OK;
  for (int32_t ipt : ipts) {
    if (!fits(b, ipt)) continue;  // a workspace sized for larger tiles
    if ((st = replan(b, ipt, stream)) != GRNG_OK) break;
    for (int32_t c : ctas) {
      b->ctas_per_sm = c;
      // tuning fills do not advance the offsets: they rewrite the same outputs
      if ((st = batch_enqueue(b, stream, false)) != GRNG_OK) break;
      cudaEventRecord(e0, stream);
      for (int k = 0; k < 3 && st == GRNG_OK; ++k) st = batch_enqueue(b, stream, false);
      cudaEventRecord(e1, stream);
      if (st != GRNG_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("batch autotune: timing failed");
        cudaGetLastError();
        st = GRNG_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 3 < best) {
        best = ms / 3;
        arg_ipt = ipt;
        arg_ctas = c;
      }
    }
    if (st != GRNG_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == GRNG_OK) st = replan(b, arg_ipt, stream);
  b->ctas_per_sm = arg_ctas;
  if (st != GRNG_OK) return st;
  if (best_ipt) *best_ipt = arg_ipt;
  if (best_ctas) *best_ctas = arg_ctas;
  if (best_ms) *best_ms = best;
  return GRNG_OK;
}

grng_status grng_batch_commit(grng_batch_t b, grng_stream_t stream) {
  if (b == nullptr) {
    set_error("batch is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::vector<uint64_t> offs(2 * (size_t)b->count);
  const char* ws = reinterpret_cast<const char*>(b->workspace);
  cudaError_t err = cudaMemcpyAsync(offs.data(), ws + b->offs_off, 16u * (size_t)b->count,
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    set_error("batch commit failed: %s", cudaGetErrorString(err));
    cudaGetLastError();
    return GRNG_ERR_CUDA;
  }
  // an engine continues where the device offset of its first request points
  // (its start plus the launches' advances): skip it ahead to that offset
  for (int32_t i = 0; i < b->count; ++i) {
    if (b->first_req_of_engine[i] != i) continue;
    grng_engine_state es;
    grng_engine_get_state(b->engines[i], &es);
    const uint64_t d_lo = offs[2 * i] - es.offset_lo;
    const uint64_t d_hi = offs[2 * i + 1] - es.offset_hi - ((offs[2 * i] < es.offset_lo) ? 1u : 0u);
    grng_engine_skip_ahead(b->engines[i], d_lo, d_hi);
  }
  return GRNG_OK;
}

grng_status grng_batch_destroy(grng_batch_t b) {
  delete b;
  return GRNG_OK;
}

}  // extern "C"
