// MRG32k3a fill kernels with the distribution transform fused in.
//
// MRG32k3a (L'Ecuyer 1999; the paper's "MRG-based generators", Sec. 4.1) is a
// sequential recursion, so the output is cut into per-thread chunks of
// consecutive units.  Each thread
//   1. jumps the call's starting state to its chunk with the compile-time
//      table of A^(2^j) in constant memory (all lanes read the same level at
//      the same time, so the reads broadcast);
//   2. steps the two component recursions in registers, with products
//      reduced by folding 2^32 = c (mod 2^32 - c) instead of dividing;
//   3. transforms each unit and writes its output words to its row of a
//      per-warp shared-memory stage (rows padded to 33 words: no bank
//      conflicts);
//   4. with its warp, copies the 32 staged rows out: 8 lanes per 128-byte
//      row with 16-byte stores when the output is 16-byte aligned, otherwise
//      one 128-byte row per instruction with 4-byte stores.
// Chunks are placed so that every chunk starts on a 16-byte output boundary
// (the first chunk of a stream has virtual head units), hence aligned rows.
// When the output's start splits a Box-Muller pair (an odd element offset
// into a 16-byte group) each chunk starts one pair earlier, with the pair
// that straddles its first 16-byte boundary, and stages its outputs shifted
// by one element (a one-element carry from pair to pair), so the rows are
// again whole 16-byte groups; the straddling pair is computed by both
// neighbouring chunks.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "device_common.cuh"
#include "grng_internal.h"
#include "mrg_tables.h"

namespace grng {

__constant__ mrg::PowTable c_mrg_pow = mrg::make_pow_table();

namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRowWords = 32;  // output words per row per sub-chunk (128 bytes)
constexpr int kJumpLevels = 24;  // per-launch jump tables: up to 2^24 chunks and streams

struct MrgParams {
  TransformParams t;
  void* out;
  int64_t n;                  // elements per stream
  int64_t units;              // units per stream
  int64_t out_words;          // output words per stream (n * es / 4)
  int64_t chunk_units;        // units per thread (multiple of 32 / wpu)
  int64_t chunks_per_stream;
  int64_t total_chunks;
  int64_t head_units;         // virtual units before `out` in the first chunk
  uint64_t stride_lo, stride_hi;  // word stride between streams
  uint32_t x[6];              // state at the call's word offset
  uint32_t x1[6];             // state at the first unit of chunk 1 of stream 0
  int32_t chunk_levels;       // entries of chunk_tab (0: generic jump)
  int32_t stream_levels;      // entries of stream_tab
  uint32_t chunk_tab[kJumpLevels][2][9];   // A^(chunk_units wpu 2^k)
  uint32_t stream_tab[kJumpLevels][2][9];  // A^(stride 2^k)
};

// p mod m for the products of one step (p < 2^54), folding 2^32 = c (mod m)
// with as few 32x32 -> 64-bit products as the ranges allow (they take twice
// the multiplier's time of a 32-bit product): m1: the high word times c1 fits
// 32 bits, so one 32-bit product, an add whose carry out is worth c1, and a
// conditional subtraction; m2: one wide fold (the high word times c2 needs
// 37 bits), then the same 32-bit step.
__device__ __forceinline__ uint32_t red_m1(uint64_t p) {
  const uint32_t lo = (uint32_t)p;
  const uint32_t u0 = lo + (uint32_t)(p >> 32) * mrg::C1;  // high word < 2^22: product < 2^30
  const uint32_t u = u0 + (u0 < lo ? mrg::C1 : 0u);        // a carry out of 2^32 is worth c1
  return u >= mrg::M1 ? u - mrg::M1 : u;
}
__device__ __forceinline__ uint32_t red_m2(uint64_t p) {
  const uint64_t t = (uint64_t)(uint32_t)p + (p >> 32) * (uint64_t)mrg::C2;  // < 2^32 + 2^37
  const uint32_t tl = (uint32_t)t;
  const uint32_t u0 = tl + (uint32_t)(t >> 32) * mrg::C2;  // t >> 32 < 2^6: product < 2^21
  const uint32_t u = u0 + (u0 < tl ? mrg::C2 : 0u);
  return u >= mrg::M2 ? u - mrg::M2 : u;
}

struct MrgRegs {
  uint32_t a0, a1, a2;  // x1_{n-3}, x1_{n-2}, x1_{n-1}
  uint32_t b0, b1, b2;  // x2_{n-3}, x2_{n-2}, x2_{n-1}
};

// One step of both components; returns z_n = (x1_n - x2_n) mod m1.
// -a13 x = a13 (m1 - x) (mod m1) keeps the sums non-negative and below 2^54.
__device__ __forceinline__ uint32_t mrg_next(MrgRegs& s) {
  const uint64_t p1 = (uint64_t)mrg::A12 * s.a1 + (uint64_t)mrg::A13 * (mrg::M1 - s.a0);
  const uint64_t p2 = (uint64_t)mrg::A21 * s.b2 + (uint64_t)mrg::A23 * (mrg::M2 - s.b0);
  const uint32_t n1 = red_m1(p1);
  const uint32_t n2 = red_m2(p2);
  s.a0 = s.a1;
  s.a1 = s.a2;
  s.a2 = n1;
  s.b0 = s.b1;
  s.b1 = s.b2;
  s.b2 = n2;
  return n1 >= n2 ? n1 - n2 : n1 - n2 + mrg::M1;
}

// y = M x mod m with one fold per product: each product p < 2^64 becomes
// (p mod 2^32) + (p >> 32) c < 2^32 (c + 1); three of them sum below 2^49,
// which two more folds and a conditional subtraction reduce.
template <uint32_t kM, uint32_t kC>
__device__ __forceinline__ uint32_t row_mod(const uint32_t* m, const uint32_t* x) {
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint64_t p = (uint64_t)m[k] * x[k];
    acc += (uint64_t)(uint32_t)p + (uint64_t)(uint32_t)(p >> 32) * kC;
  }
  const uint64_t t = (uint64_t)(uint32_t)acc + (uint64_t)(uint32_t)(acc >> 32) * kC;
  const uint64_t u = (uint64_t)(uint32_t)t + (uint64_t)(uint32_t)(t >> 32) * kC;
  const uint32_t v = (uint32_t)u + (uint32_t)(u >> 32) * kC;
  return v >= kM ? v - kM : v;
}

__device__ __forceinline__ void apply(const uint32_t* m1, const uint32_t* m2, MrgRegs& s) {
  const uint32_t x1[3] = {s.a0, s.a1, s.a2};
  const uint32_t x2[3] = {s.b0, s.b1, s.b2};
  s.a0 = row_mod<mrg::M1, mrg::C1>(m1 + 0, x1);
  s.a1 = row_mod<mrg::M1, mrg::C1>(m1 + 3, x1);
  s.a2 = row_mod<mrg::M1, mrg::C1>(m1 + 6, x1);
  s.b0 = row_mod<mrg::M2, mrg::C2>(m2 + 0, x2);
  s.b1 = row_mod<mrg::M2, mrg::C2>(m2 + 3, x2);
  s.b2 = row_mod<mrg::M2, mrg::C2>(m2 + 6, x2);
}

// Applies table[k] (= A^(unit 2^k), both components) for the set bits of e;
// the loop over levels is warp-uniform so all lanes read the same entry.
__device__ __forceinline__ void jump_table(MrgRegs& s, const uint32_t (*tab)[2][9], int levels,
                                           uint64_t e) {
  for (int k = 0; k < levels; ++k) {
    if ((e >> k) & 1u) apply(tab[k][0], tab[k][1], s);
    if (!__any_sync(0xFFFFFFFFu, (e >> k) > 1u)) break;
  }
}

__device__ __forceinline__ void jump(MrgRegs& s, uint64_t e_lo, uint64_t e_hi) {
  uint32_t x1[3] = {s.a0, s.a1, s.a2};
  uint32_t x2[3] = {s.b0, s.b1, s.b2};
  // Uniform loop over levels so that all lanes read the same table entry.
  for (int j = 0; j < mrg::kLevels; ++j) {
    const uint64_t word = j < 64 ? e_lo : e_hi;
    const bool bit = (word >> (j & 63)) & 1u;
    if (bit) {
      mrg::matvec(c_mrg_pow.m[0][j], x1, mrg::M1, mrg::C1);
      mrg::matvec(c_mrg_pow.m[1][j], x2, mrg::M2, mrg::C2);
    }
    // stop once no lane has bits left at or above j + 1
    const uint64_t rest_lo = j + 1 < 64 ? (e_lo >> (j + 1)) : 0;
    const uint64_t rest_hi = j + 1 < 64 ? e_hi : (j + 1 < 128 ? (e_hi >> ((j + 1) & 63)) : 0);
    if (!__any_sync(0xFFFFFFFFu, (rest_lo | rest_hi) != 0)) break;
  }
  s.a0 = x1[0]; s.a1 = x1[1]; s.a2 = x1[2];
  s.b0 = x2[0]; s.b1 = x2[1]; s.b2 = x2[2];
}

// Generates one unit's words and writes its kWpu output words to o.
template <int V>
__device__ __forceinline__ void gen_unit(MrgRegs& st, uint32_t* o, const TransformParams& t,
                                         bool odd = false) {
  constexpr int kWpu = VInfo<V>::wpu;
  uint32_t w[kWpu];
#pragma unroll
  for (int i = 0; i < kWpu; ++i) w[i] = mrg_next(st);
  unit_outputs<V>(w, o, t, odd);
}

// The 16-byte stage chunk from 4 new output words: as they are, or (carry
// mode) shifted up by one element of kOwpe words behind the carried element,
// whose place the new last element takes.
template <bool kCarry, int kOwpe>
__device__ __forceinline__ uint4 shift_in(uint32_t* carry, const uint32_t* o4) {
  if constexpr (!kCarry) {
    return make_uint4(o4[0], o4[1], o4[2], o4[3]);
  } else if constexpr (kOwpe == 1) {
    const uint4 v = make_uint4(carry[0], o4[0], o4[1], o4[2]);
    carry[0] = o4[3];
    return v;
  } else {
    const uint4 v = make_uint4(carry[0], carry[1], o4[0], o4[1]);
    carry[0] = o4[2];
    carry[1] = o4[3];
    return v;
  }
}

// kMode: 0 output not 16-byte alignable (row-by-row 4-byte copy-out);
// 1 chunks start on 16-byte boundaries at unit boundaries; 2 chunks start on
// 16-byte boundaries one element into a Box-Muller pair (carry mode);
// 3 substreams of unequal 16-byte phase: each stream has its own head, and
// its own carry mode when its start splits a pair (a warp's 32 chunks lie in
// one stream, so both are warp-uniform).
template <int V, int kMode>
__global__ void __launch_bounds__(kThreads) mrg_fill_kernel(const MrgParams p) {
  constexpr bool kAligned = kMode != 0;
  constexpr bool kPerStream = kMode == 3;
  constexpr int kWpu = VInfo<V>::wpu;
  constexpr int kOwpe = VInfo<V>::ow_per_elem;
  constexpr int kSu = kRowWords / kWpu;  // units per sub-chunk
  // per warp: 32 rows (one per lane) of 8 16-byte chunks; chunk q of row r is
  // kept at position q ^ (r & 7), so a lane's chunk stores and the copy-out's
  // row loads are both free of bank conflicts
  __shared__ uint4 stage[kWarps][32][8];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t cid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool active = cid < p.total_chunks;
  int64_t s = 0, c = 0;
  if (active) {
    s = cid / p.chunks_per_stream;
    c = cid - s * p.chunks_per_stream;
  }
  // the stream's head (virtual units before its output's first 16-byte
  // group) and whether its start splits a pair
  int64_t hu = p.head_units;
  bool kCarry = kMode == 2;
  if constexpr (kPerStream) {
    const uint32_t he = (uint32_t)(((uintptr_t)p.out + (uintptr_t)(s * p.n * VInfo<V>::es)) &
                                   15u) /
                        (uint32_t)VInfo<V>::es;
    constexpr uint32_t kEpu = (uint32_t)VInfo<V>::epu;
    hu = (int64_t)((he + kEpu - 1) / kEpu);
    kCarry = kEpu == 2 && (he & 1u) != 0;
  }
  const int64_t u_first = c * p.chunk_units - hu;

  MrgRegs st;
  if (p.chunk_levels > 0) {
    // chunk 0 starts at the call's state, chunk c >= 1 at chunk 1's state
    // jumped by c - 1 chunks; then stream s jumps by s strides
    const uint32_t* x = c == 0 ? p.x : p.x1;
    st.a0 = x[0]; st.a1 = x[1]; st.a2 = x[2];
    st.b0 = x[3]; st.b1 = x[4]; st.b2 = x[5];
    jump_table(st, p.chunk_tab, p.chunk_levels, active && c > 0 ? (uint64_t)(c - 1) : 0u);
    if (p.stream_levels > 0) jump_table(st, p.stream_tab, p.stream_levels, active ? (uint64_t)s : 0u);
    if constexpr (kPerStream) {
      // chunk 1's state is taken at the largest head (p.head_units); a stream
      // with a smaller head starts its chunks that many units later
      if (active && c > 0)
        for (int64_t k = 0; k < (p.head_units - hu) * kWpu; ++k) mrg_next(st);
    }
  } else {
    st.a0 = p.x[0]; st.a1 = p.x[1]; st.a2 = p.x[2];
    st.b0 = p.x[3]; st.b1 = p.x[4]; st.b2 = p.x[5];
    // words to skip: s * stride + max(u_first, 0) * wpu  (mod 2^128)
    uint64_t e_lo = 0, e_hi = 0;
    if (active) {
      const uint64_t us = (uint64_t)s;
      e_lo = us * p.stride_lo;
      e_hi = __umul64hi(us, p.stride_lo) + us * p.stride_hi;
      const uint64_t add = (uint64_t)((u_first > 0 ? u_first : 0) * kWpu);
      const uint64_t sum = e_lo + add;
      e_hi += (sum < e_lo) ? 1u : 0u;
      e_lo = sum;
    }
    jump(st, e_lo, e_hi);
  }

  // carry mode: the chunk's first unit straddles its first 16-byte boundary;
  // only its second element is output here (the previous chunk outputs the
  // first), and every later element moves up one place
  uint32_t carry[kOwpe];
  if (kCarry) {
    uint32_t o[kWpu];
#pragma unroll
    for (int i = 0; i < kWpu; ++i) o[i] = 0u;
    if (active && u_first >= 0 && u_first < p.units) gen_unit<V>(st, o, p.t);
#pragma unroll
    for (int i = 0; i < kOwpe; ++i) carry[i] = o[kOwpe + i];
  }
  const int64_t nsub = p.chunk_units / kSu;
  uint32_t* out_words = reinterpret_cast<uint32_t*>(p.out);
  // Aligned copy-out: lane copies 16-byte piece (lane & 7) of rows
  // it * 4 + (lane >> 3), it = 0..7.  The host makes chunks_per_stream a
  // multiple of 32 when there are several streams, so the 32 chunks of a
  // warp lie in one stream and row r is chunk cw + r of that stream.
  const int64_t cw = ((int64_t)blockIdx.x * kThreads + warp * 32);  // warp's first chunk id
  const int64_t sw = cw / p.chunks_per_stream;
  const int64_t cw_in = cw - sw * p.chunks_per_stream;
  const int64_t lim_chunks = (sw + 1) * p.chunks_per_stream < p.total_chunks
                                 ? (sw + 1) * p.chunks_per_stream
                                 : p.total_chunks;
  const int rows_active = (int)((lim_chunks - cw) < 32 ? (lim_chunks - cw) : 32);
  const int64_t row_stride = 4 * p.chunk_units * kWpu;  // words between rows it and it + 1
  const int64_t ow_lane = ((cw_in + (lane >> 3)) * p.chunk_units - hu) * kWpu +
                          (kCarry ? kOwpe : 0) + (lane & 7) * 4;
  uint32_t* stream_out = out_words + sw * p.out_words;
  for (int64_t q = 0; q < nsub; ++q) {
    // first unit of this sub-chunk (in carry mode after the straddling one)
    const int64_t ub = u_first + (kCarry ? 1 : 0) + q * kSu;
    constexpr int kUpc = 4 / kWpu;          // units per 16-byte chunk
    if (active) {
      if (ub >= 0 && ub + kSu <= p.units) {
        constexpr int kChUnroll = VInfo<V>::weight == 0 ? 8 : VInfo<V>::weight == 1 ? 2 : 1;
#pragma unroll kChUnroll
        for (int ch = 0; ch < 8; ++ch) {
          uint32_t o4[4];
#pragma unroll
          for (int u = 0; u < kUpc; ++u) gen_unit<V>(st, o4 + u * kWpu, p.t, (u & 1) != 0);
          stage[warp][lane][ch ^ (lane & 7)] = kCarry ? shift_in<true, kOwpe>(carry, o4)
                                                      : shift_in<false, kOwpe>(carry, o4);
        }
      } else {
        for (int ch = 0; ch < 8; ++ch) {
          uint32_t o4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
          for (int u = 0; u < kUpc; ++u) {
            const int64_t unit = ub + ch * kUpc + u;
            if (unit >= 0 && unit < p.units) gen_unit<V>(st, o4 + u * kWpu, p.t);
          }
          stage[warp][lane][ch ^ (lane & 7)] = kCarry ? shift_in<true, kOwpe>(carry, o4)
                                                      : shift_in<false, kOwpe>(carry, o4);
        }
      }
    }
    __syncwarp();
    if constexpr (kAligned) {
      // interior sub-chunks (every row present and inside the stream, the
      // common case) store without per-row checks
      const int64_t ow0 = ow_lane + q * kRowWords;
      const bool inside = ow0 >= 0 && ow0 + 7 * row_stride + 4 <= p.out_words;
      if (__all_sync(0xFFFFFFFFu, inside && rows_active == 32)) {
        uint32_t* dst = stream_out + ow0;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int r = it * 4 + (lane >> 3);
          store16(dst + it * row_stride, stage[warp][r][(lane & 7) ^ (r & 7)]);
        }
        __syncwarp();
        continue;
      }
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int r = it * 4 + (lane >> 3);
        if (r >= rows_active) continue;
        const int64_t ow = ow_lane + it * row_stride + q * kRowWords;
        const uint4 v = stage[warp][r][(lane & 7) ^ (r & 7)];
        if (ow >= 0 && ow + 4 <= p.out_words) {
          store16(stream_out + ow, v);
        } else {
          const uint32_t src[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (ow + i >= 0 && ow + i < p.out_words) stream_out[ow + i] = src[i];
        }
      }
    } else {
      const uint32_t s_lo = (uint32_t)s, s_hi = (uint32_t)((uint64_t)s >> 32);
      const uint32_t ub_lo = (uint32_t)ub, ub_hi = (uint32_t)((uint64_t)ub >> 32);
      for (int r = 0; r < 32; ++r) {
        const bool r_active = __shfl_sync(0xFFFFFFFFu, active ? 1 : 0, r) != 0;
        const int64_t r_s = (int64_t)(((uint64_t)__shfl_sync(0xFFFFFFFFu, s_hi, r) << 32) |
                                      __shfl_sync(0xFFFFFFFFu, s_lo, r));
        const int64_t r_ub = (int64_t)(((uint64_t)__shfl_sync(0xFFFFFFFFu, ub_hi, r) << 32) |
                                       __shfl_sync(0xFFFFFFFFu, ub_lo, r));
        if (!r_active) continue;
        const int64_t ow = r_ub * kWpu + lane;
        const uint32_t* chunk =
            reinterpret_cast<const uint32_t*>(&stage[warp][r][(lane >> 2) ^ (r & 7)]);
        if (ow >= 0 && ow < p.out_words) out_words[r_s * p.out_words + ow] = chunk[lane & 3];
      }
    }
    __syncwarp();
  }
}

// Host matrix arithmetic for the per-launch tables (3x3 mod m, row-major).
constexpr mrg::PowTable kHostPow = mrg::make_pow_table();

void host_matmul(const uint32_t* a, const uint32_t* b, uint32_t* out, uint32_t m) {
  uint32_t r[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      unsigned __int128 acc = 0;
      for (int k = 0; k < 3; ++k) acc += (unsigned __int128)a[3 * i + k] * b[3 * k + j];
      r[3 * i + j] = (uint32_t)(acc % m);
    }
  std::memcpy(out, r, sizeof(r));
}

// A_c^e for a 128-bit exponent from the A^(2^j) table.
void host_pow(int comp, uint64_t e_lo, uint64_t e_hi, uint32_t* out) {
  const uint32_t m = comp == 0 ? mrg::M1 : mrg::M2;
  uint32_t r[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  for (int j = 0; j < 128; ++j) {
    const uint64_t w = j < 64 ? e_lo : e_hi;
    if ((w >> (j & 63)) & 1u) host_matmul(r, kHostPow.m[comp][j], r, m);
  }
  std::memcpy(out, r, sizeof(r));
}

// tab[k] = A^(e 2^k) for k < levels (both components).
void host_table(uint64_t e_lo, uint64_t e_hi, int levels, uint32_t (*tab)[2][9]) {
  for (int c = 0; c < 2; ++c) {
    const uint32_t m = c == 0 ? mrg::M1 : mrg::M2;
    uint32_t a[9];
    host_pow(c, e_lo, e_hi, a);
    for (int k = 0; k < levels; ++k) {
      std::memcpy(tab[k][c], a, sizeof(a));
      host_matmul(a, a, a, m);
    }
  }
}

int bits_for(int64_t v) {  // number of bits to represent v >= 0
  int b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

template <int V>
grng_status launch_variant(const FillRequest& r, cudaStream_t stream) {
  using I = VInfo<V>;
  constexpr int kSu = kRowWords / I::wpu;
  int dev = 0;
  const int sms = current_device_sms(&dev);
  MrgParams p;
  p.t = r.t;
  p.out = r.out;
  p.n = r.n;
  p.units = (r.n + I::epu - 1) / I::epu;
  p.out_words = r.n * (I::es / 4);
  p.stride_lo = r.stride_lo;
  p.stride_hi = r.stride_hi;
  for (int i = 0; i < 6; ++i) p.x[i] = r.mrg[i];

  const uintptr_t addr = (uintptr_t)r.out;
  const uint32_t phase_w = (uint32_t)((addr & 15u) / 4u);
  const uint64_t stream_bytes = (uint64_t)r.n * I::es;
  const bool uniform_streams = r.num_streams == 1 || (stream_bytes % 16u) == 0;
  const bool aligned = uniform_streams && (phase_w % (uint32_t)I::wpu) == 0;
  // a Box-Muller pair split by the output's start: head elements odd
  const int64_t head_e = (int64_t)(phase_w * 4u / I::es);
  const bool carry = uniform_streams && !aligned && I::epu == 2 && (head_e & 1) != 0;
  // substreams of unequal phase: per-stream heads up to the largest possible
  // one, ceil((16 / es - 1) / epu) units
  const bool per_stream = !uniform_streams;
  const int64_t hu_max = (16 / I::es - 1 + I::epu - 1) / I::epu;
  p.head_units = aligned ? (int64_t)(phase_w / I::wpu)
                 : carry ? (head_e + 1) / 2
                 : per_stream ? hu_max : 0;

  // About one resident wave of threads, one chunk each (2048 threads per SM,
  // or the tuned count).
  const int32_t geom = fill_geometry(GRNG_MRG32K3A, V, r.n * r.num_streams);
  const int64_t target_threads = (int64_t)sms * (geom > 0 ? 256 * (int64_t)geom : 2048);
  int64_t per_stream_threads = target_threads / r.num_streams;
  if (per_stream_threads < 1) per_stream_threads = 1;
  const int64_t span = p.units + p.head_units;
  int64_t cu = (span + per_stream_threads - 1) / per_stream_threads;
  if (cu < 2 * kSu) cu = 2 * kSu;
  cu = (cu + kSu - 1) / kSu * kSu;
  int64_t cps = (span + cu - 1) / cu;
  if (r.num_streams > 1) {
    // a multiple of 32 chunks per stream keeps each warp's 32 chunks inside
    // one stream; the units are spread over all of them
    cps = (cps + 31) / 32 * 32;
    cu = (span + cps - 1) / cps;
    cu = (cu + kSu - 1) / kSu * kSu;
  }
  p.chunk_units = cu;
  p.chunks_per_stream = cps;
  p.total_chunks = p.chunks_per_stream * r.num_streams;
  // per-launch jump tables (chunk-granular and stream-granular exponents)
  const int clev = bits_for(cps - 1), slev = bits_for(r.num_streams - 1);
  p.chunk_levels = 0;
  p.stream_levels = 0;
  if (clev <= kJumpLevels && slev <= kJumpLevels && cps > 1) {
    static thread_local struct {
      bool valid = false;
      uint64_t cw, s_lo, s_hi;
      int clev, slev;
      uint32_t ctab[kJumpLevels][2][9], stab[kJumpLevels][2][9];
    } cache;
    const uint64_t cw = (uint64_t)cu * I::wpu;
    if (!(cache.valid && cache.cw == cw && cache.clev >= clev &&
          (slev == 0 || (cache.s_lo == r.stride_lo && cache.s_hi == r.stride_hi && cache.slev >= slev)))) {
      host_table(cw, 0, clev, cache.ctab);
      if (slev > 0) host_table(r.stride_lo, r.stride_hi, slev, cache.stab);
      cache.valid = true;
      cache.cw = cw;
      cache.s_lo = r.stride_lo;
      cache.s_hi = r.stride_hi;
      cache.clev = clev;
      cache.slev = slev;
    }
    std::memcpy(p.chunk_tab, cache.ctab, sizeof(p.chunk_tab));
    std::memcpy(p.stream_tab, cache.stab, sizeof(p.stream_tab));
    p.chunk_levels = clev;
    p.stream_levels = slev;
    // state at the first unit of chunk 1: (cu - head) units after the call's offset
    uint32_t a[9], b[9];
    const uint64_t e = (uint64_t)(cu - p.head_units) * I::wpu;
    host_pow(0, e, 0, a);
    host_pow(1, e, 0, b);
    for (int i = 0; i < 3; ++i) {
      uint64_t acc1 = 0, acc2 = 0;
      for (int k = 0; k < 3; ++k) {
        acc1 = (acc1 + (uint64_t)a[3 * i + k] * r.mrg[k] % mrg::M1) % mrg::M1;
        acc2 = (acc2 + (uint64_t)b[3 * i + k] * r.mrg[3 + k] % mrg::M2) % mrg::M2;
      }
      p.x1[i] = (uint32_t)acc1;
      p.x1[3 + i] = (uint32_t)acc2;
    }
  }
  const int64_t grid = (p.total_chunks + kThreads - 1) / kThreads;
  if (grid > 0x7FFFFFFF) {
    set_error("MRG32k3a fill: grid too large");
    return GRNG_ERR_UNSUPPORTED;
  }
  if (aligned) {
    mrg_fill_kernel<V, 1><<<(unsigned)grid, kThreads, 0, stream>>>(p);
  } else if (carry) {
    if constexpr (I::epu == 2) mrg_fill_kernel<V, 2><<<(unsigned)grid, kThreads, 0, stream>>>(p);
  } else if (per_stream) {
    mrg_fill_kernel<V, 3><<<(unsigned)grid, kThreads, 0, stream>>>(p);
  } else {
    mrg_fill_kernel<V, 0><<<(unsigned)grid, kThreads, 0, stream>>>(p);
  }
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error("MRG32k3a fill launch failed: %s", cudaGetErrorString(err));
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}

}  // namespace

grng_status launch_mrg(const FillRequest& r, CUstream_st* stream) {
  switch (r.variant) {
    case V_BITS: return launch_variant<V_BITS>(r, stream);
    case V_U01_F32: return launch_variant<V_U01_F32>(r, stream);
    case V_UNI_F32: return launch_variant<V_UNI_F32>(r, stream);
    case V_U01_F64: return launch_variant<V_U01_F64>(r, stream);
    case V_AFF_F64: return launch_variant<V_AFF_F64>(r, stream);
    case V_UNI_F64: return launch_variant<V_UNI_F64>(r, stream);
    case V_GAUSS_F32: return launch_variant<V_GAUSS_F32>(r, stream);
    case V_LOGN_F32: return launch_variant<V_LOGN_F32>(r, stream);
    case V_GAUSS_F64: return launch_variant<V_GAUSS_F64>(r, stream);
    case V_LOGN_F64: return launch_variant<V_LOGN_F64>(r, stream);
    case V_ICDF_GAUSS_F32: return launch_variant<V_ICDF_GAUSS_F32>(r, stream);
    case V_ICDF_LOGN_F32: return launch_variant<V_ICDF_LOGN_F32>(r, stream);
    case V_ICDF_GAUSS_F64: return launch_variant<V_ICDF_GAUSS_F64>(r, stream);
    case V_ICDF_LOGN_F64: return launch_variant<V_ICDF_LOGN_F64>(r, stream);
    case V_STDGAUSS_F64: return launch_variant<V_STDGAUSS_F64>(r, stream);
    default: set_error("unknown variant %d", r.variant); return GRNG_ERR_INVALID_ARG;
  }
}

}  // namespace grng
