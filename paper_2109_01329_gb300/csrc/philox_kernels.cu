// Philox4x32-10 fill kernels with the distribution transform fused in.
//
// The paper's path is two kernels: the vendor generator writes raw uniforms,
// then a SYCL kernel re-reads and rewrites the buffer to apply the range
// (Sec. 4.3, Listings 1 and 2; profiled as separate kernels in Sec. 7, Fig. 4).
// Here one kernel computes each counter block in registers, transforms it and
// stores it once: 4 output bytes per word and no reads.
//
// Output is cut into 16-byte groups at 16-byte aligned addresses.  Every
// variant consumes exactly 4 words per 16 output bytes, so:
//   * stream / multi kernels: when the word phase of the first group matches
//     its block boundary (and Box-Muller pairs do not straddle groups), group
//     j is exactly Philox block base + j: one block, one transform, one
//     st.v4.  Only the first and the last group of a stream may be partial.
//   * shift kernel (one stream at any other phase): group j is the tail of
//     block base + j and the head of block base + j + 1; a warp computes 32
//     consecutive blocks and emits 31 groups, exchanging the words between
//     neighbouring lanes by shuffle.  When the output's start splits a
//     Box-Muller pair, lanes transform pair-aligned groups one element
//     earlier and exchange the straddling element too (30 groups per warp).
//   * rotate kernel (one stream of 2- or 4-word units at a word offset
//     that keeps them inside blocks, the output start at another 16-byte
//     phase): each lane transforms its own block and rotates its outputs
//     into the group that lane - 1's block opens, by shuffle; lane 0 and
//     lane 31 write the groups shared with the neighbouring warps' chunks
//     with narrower stores, so no unit is transformed twice.
//   * multi-shift kernel: substreams at another phase or alignment, the
//     shift kernel's exchange applied per stream (a warp works on 30 groups
//     of one stream).
// Both write every output exactly once; results do not depend on the launch
// geometry (each output is a function of its word index only).
#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>

#include "device_common.cuh"
#include "grng_internal.h"

namespace grng {
namespace {

using namespace dev;

constexpr int kThreads = 256;

__device__ __forceinline__ void add128(uint64_t& lo, uint64_t& hi, uint64_t vlo, uint64_t vhi) {
  const uint64_t s = lo + vlo;
  hi += vhi + ((s < lo) ? 1u : 0u);
  lo = s;
}

// Stores the in-range elements of a partial group whose first element is e0.
template <int V>
__device__ __forceinline__ void store_partial(char* stream_base, int64_t e0, int64_t n, uint4 o) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  const uint32_t ow[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
  for (int i = 0; i < kEpg; ++i) {
    const int64_t e = e0 + i;
    if (e >= 0 && e < n) {
      if constexpr (I::es == 4) {
        reinterpret_cast<uint32_t*>(stream_base)[e] = ow[i];
      } else {
        reinterpret_cast<uint2*>(stream_base)[e] = make_uint2(ow[2 * i], ow[2 * i + 1]);
      }
    }
  }
}

// ------------------------------------------------------------ single stream
// Full 16-byte groups [jf, jl) in the main loop, U independent counter blocks
// per thread per iteration (stores of the U blocks are each coalesced across
// the warp), pointer and counter advanced by increments.  The at most two
// partial groups (the first and the last) are done by the grid's first two
// threads before the loop.
struct StreamParams {
  TransformParams t;
  uint4* gbase;       // 16-byte aligned address of group 0 (may precede out)
  void* out;
  int64_t n;          // elements
  int64_t head;       // elements of group 0 that lie before out
  int64_t jf, jl;     // full groups [jf, jl)
  int64_t edge[2];    // partial groups, or -1
  uint64_t base_lo;   // block counter of group 0
  uint64_t base_hi;
  PhiloxRoundKeys rk;
};

template <int V, bool kHiUniform>
__device__ __forceinline__ uint4 group_block(const StreamParams& p, uint64_t j) {
  const uint64_t lo = p.base_lo + j;
  const uint64_t hi = kHiUniform ? p.base_hi : p.base_hi + ((lo < p.base_lo) ? 1u : 0u);
  return philox4x32_10(ctr_from(lo, hi), p.rk);
}

template <int V, int U, bool kHiUniform>
__device__ __forceinline__ void philox_stream_body(const StreamParams& p) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  const int64_t T = (int64_t)gridDim.x * kThreads;
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (tid < 2 && p.edge[tid] >= 0) {
    const int64_t j = p.edge[tid];
    const uint4 o = block_outputs<V>(group_block<V, false>(p, (uint64_t)j), p.t);
    store_partial<V>(reinterpret_cast<char*>(p.out), j * kEpg - p.head, p.n, o);
  }
  int64_t j = p.jf + tid;
  uint4* dst = p.gbase + j;
  for (; j + (U - 1) * T < p.jl; j += U * T, dst += U * T) {
    uint4 o[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      o[u] = block_outputs<V>(group_block<V, kHiUniform>(p, (uint64_t)(j + u * T)), p.t);
#pragma unroll
    for (int u = 0; u < U; ++u) dst[u * T] = o[u];
  }
  for (; j < p.jl; j += T, dst += T)
    *dst = block_outputs<V>(group_block<V, kHiUniform>(p, (uint64_t)j), p.t);
}

// Counter blocks per thread per loop iteration: six for bits and the FP32
// uniforms (2, 4, 6 and 8 measured: 6 fastest), two for the other FP32 and
// the FP64 uniform transforms (3 and 4 slower), one for the FP64 fixed-point
// transforms (hundreds of instructions per unit).
template <int V>
constexpr int blocks_per_thread() {
  return (V == V_BITS || V == V_U01_F32 || V == V_UNI_F32) ? 6
         : (V == V_GAUSS_F64 || V == V_LOGN_F64 || V == V_STDGAUSS_F64 ||
            V == V_ICDF_GAUSS_F64 || V == V_ICDF_LOGN_F64)
             ? 1
             : 2;
}

// The Box-Muller and FP32 inverse-CDF variants gain from a fifth resident CTA
// per SM (registers capped near 51: 1-5 % faster); the light variants keep
// the compiler's own register choice, which a CTA minimum would change.
template <int V>
constexpr bool stream_wants_5_ctas() {
  return V == V_GAUSS_F32 || V == V_LOGN_F32 || V == V_ICDF_GAUSS_F32 || V == V_GAUSS_F64 ||
         V == V_STDGAUSS_F64 || V == V_LOGN_F64 || V == V_ICDF_GAUSS_F64 || V == V_ICDF_LOGN_F64;
}

template <int V, int U, bool kHiUniform>
__global__ void __launch_bounds__(kThreads) philox_stream_kernel(const __grid_constant__ StreamParams p) {
  philox_stream_body<V, U, kHiUniform>(p);
}

template <int V, int U, bool kHiUniform>
__global__ void __launch_bounds__(kThreads, 5) philox_stream_kernel_5(const __grid_constant__ StreamParams p) {
  philox_stream_body<V, U, kHiUniform>(p);
}

// ------------------------------------------------------ single stream, shifted
// The same groups when the word offset is not on a block boundary (phase
// ph = 1..3 after removing the head words): group j is the last 4 - ph words
// of block base + j and the first ph words of block base + j + 1.  Each warp
// computes 32 consecutive blocks and emits the 31 groups that start in its
// lanes 0..30, taking the next block's words from lane + 1 by shuffle, so a
// group still costs 32/31 of a block and no shared memory or barrier.  U
// chunks of groups per warp per iteration, as U blocks per thread above.
//
// kSplit: the output's start splits a Box-Muller pair (odd head).  Lane l
// then transforms the pair-aligned "virtual" group that starts one element
// earlier (its words found as above, for any phase), and output group j is
// virtual group j without its first element plus the first element of
// virtual group j + 1, taken from lane + 1: 30 groups per warp, every pair
// transformed once.
struct ShiftParams {
  TransformParams t;
  uint4* gbase;       // 16-byte aligned address of group 0 (may precede out)
  void* out;
  int64_t n;          // elements
  int64_t head;       // elements of group 0 that lie before out
  int64_t groups;
  int64_t jf, jl;     // groups [jf, jl) lie wholly inside the output
  int64_t chunks;     // ceil(groups / groups per warp chunk)
  uint64_t base_lo;   // block holding the first word of (virtual) group 0
  uint64_t base_hi;
  uint32_t ph;        // its word phase: 1..3, or 0..3 with kSplit
  PhiloxRoundKeys rk;
};

template <bool kSplit>
__host__ __device__ constexpr int shift_per_warp() {
  return kSplit ? 30 : 31;
}

// The 4 words of a group whose first word is at phase kPh (1..3) of block b
// (this lane's), the rest from the next lane's block; kPh a constant, so only
// the kPh words needed cross lanes.
template <int kPh>
__device__ __forceinline__ uint4 shift_words_c(uint4 b) {
  const uint32_t n0 = __shfl_down_sync(0xFFFFFFFFu, b.x, 1);
  if constexpr (kPh == 1) {
    return make_uint4(b.y, b.z, b.w, n0);
  } else {
    const uint32_t n1 = __shfl_down_sync(0xFFFFFFFFu, b.y, 1);
    if constexpr (kPh == 2) {
      return make_uint4(b.z, b.w, n0, n1);
    } else {
      const uint32_t n2 = __shfl_down_sync(0xFFFFFFFFu, b.z, 1);
      return make_uint4(b.w, n0, n1, n2);
    }
  }
}

// The same with the phase ph known only at run time (warp-uniform).
__device__ __forceinline__ uint4 shift_words(uint4 b, uint32_t ph) {
  const uint32_t n0 = __shfl_down_sync(0xFFFFFFFFu, b.x, 1);
  const uint32_t n1 = __shfl_down_sync(0xFFFFFFFFu, b.y, 1);
  const uint32_t n2 = __shfl_down_sync(0xFFFFFFFFu, b.z, 1);
  if (ph == 1) return make_uint4(b.y, b.z, b.w, n0);
  if (ph == 2) return make_uint4(b.z, b.w, n0, n1);
  if (ph == 3) return make_uint4(b.w, n0, n1, n2);
  return b;
}

// Output group from this lane's transformed virtual group v and the next
// lane's first element (a Box-Muller pair split by the output's start).
template <int V>
__device__ __forceinline__ uint4 split_group(uint4 v) {
  const uint32_t m0 = __shfl_down_sync(0xFFFFFFFFu, v.x, 1);
  const uint32_t m1 = __shfl_down_sync(0xFFFFFFFFu, v.y, 1);
  return VInfo<V>::es == 4 ? make_uint4(v.y, v.z, v.w, m0) : make_uint4(v.z, v.w, m0, m1);
}

// kPh: the word phase as a constant (1..3), or -1 to read it from p.ph.
template <int V, int U, bool kHiUniform, bool kSplit, int kPh>
__device__ __forceinline__ void philox_shift_body(const ShiftParams& p) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  constexpr int kPer = shift_per_warp<kSplit>();
  const int lane = threadIdx.x & 31;
  const int64_t TW = (int64_t)gridDim.x * (kThreads / 32);
  const int64_t c0 = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  // this lane's group of chunk c is j = c kPer + lane; j, the block counter
  // and the store address advance by increments (dj from chunk c to c + TW)
  const int64_t dj = TW * kPer;
  int64_t j = c0 * kPer + lane;
  uint64_t lo = p.base_lo + (uint64_t)j;
  uint4* dst = p.gbase + j;
  // the loop bound depends only on the warp: every shuffle has all 32 lanes
  for (int64_t c = c0; c < p.chunks;
       c += U * TW, j += U * dj, lo += (uint64_t)(U * dj), dst += U * dj) {
    uint4 b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t l = lo + (uint64_t)(u * dj);
      const uint64_t h = kHiUniform ? p.base_hi : p.base_hi + ((l < p.base_lo) ? 1u : 0u);
      b[u] = philox4x32_10(ctr_from(l, h), p.rk);
    }
    // every group of this iteration lies wholly inside the output (uniform)
    const bool interior = c * kPer >= p.jf && (c + (U - 1) * TW) * kPer + kPer <= p.jl;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uint4 w;
      if constexpr (kPh < 0) {
        w = shift_words(b[u], p.ph);
      } else {
        w = shift_words_c<kPh>(b[u]);
      }
      // every lane transforms its (virtual) group; in split mode lane l + 1's
      // first element is needed by lane l
      uint4 o = block_outputs<V>(w, p.t);
      if constexpr (kSplit) o = split_group<V>(o);
      if (interior) {
        if (lane < kPer) dst[u * dj] = o;
      } else {
        const int64_t ju = j + u * dj;
        if (lane < kPer && ju < p.groups) {
          const int64_t e0 = ju * kEpg - p.head;
          if (e0 >= 0 && e0 + kEpg <= p.n) {
            dst[u * dj] = o;
          } else {
            store_partial<V>(reinterpret_cast<char*>(p.out), e0, p.n, o);
          }
        }
      }
    }
  }
}

// The phase is the same for the whole grid.  Raw bits take one loop per
// phase, each with the phase a constant (n = 10^9 at phases 1, 2, 3: 0.764,
// 0.771, 0.796 ms against 0.852, 0.851, 0.915 with the phase a variable).  The
// FP32 uniforms take the constant form for phases 2 and 3 only: with a
// constant phase 1 they ran 10 % slower (ncu: 207 against 186 million
// instructions, the words moved into place one by one where the variable form
// selects each into place), while phases 2 and 3 gained 4-8 %.  The other
// variants keep the variable phase.
template <int V, int U, bool kHiUniform, bool kSplit>
__device__ __forceinline__ void philox_shift_phases(const ShiftParams& p) {
  if constexpr (V == V_BITS && !kSplit) {
    switch (p.ph) {
      case 1: philox_shift_body<V, U, kHiUniform, kSplit, 1>(p); break;
      case 2: philox_shift_body<V, U, kHiUniform, kSplit, 2>(p); break;
      default: philox_shift_body<V, U, kHiUniform, kSplit, 3>(p); break;
    }
  } else if constexpr ((V == V_U01_F32 || V == V_UNI_F32) && !kSplit) {
    switch (p.ph) {
      case 2: philox_shift_body<V, U, kHiUniform, kSplit, 2>(p); break;
      case 3: philox_shift_body<V, U, kHiUniform, kSplit, 3>(p); break;
      default: philox_shift_body<V, U, kHiUniform, kSplit, -1>(p); break;
    }
  } else {
    philox_shift_body<V, U, kHiUniform, kSplit, -1>(p);
  }
}

template <int V, int U, bool kHiUniform, bool kSplit>
__global__ void __launch_bounds__(kThreads) philox_shift_kernel(const __grid_constant__ ShiftParams p) {
  philox_shift_phases<V, U, kHiUniform, kSplit>(p);
}

template <int V, int U, bool kHiUniform, bool kSplit>
__global__ void __launch_bounds__(kThreads, 5) philox_shift_kernel_5(const __grid_constant__ ShiftParams p) {
  philox_shift_phases<V, U, kHiUniform, kSplit>(p);
}

// ------------------------------------------------------ single stream, rotated
// One stream whose units lie inside counter blocks (the word offset a multiple
// of the words per unit) while its output start is not at the blocks' 16-byte
// phase.  Block j's four output words are then output words 4 j - r .. 4 j -
// r + 3 (r = word offset mod 4): the last kS = (h - r) mod 4 of them open the
// next 16-byte group (h: output words of out's group before out).  Each lane
// transforms its own block once and completes its group from the last kS
// output words of lane - 1 by shuffle; lane 0 writes only its own part of its
// group and lane 31 the opening words of the next group, with 4- or 8-byte
// stores at constant offsets from the group's address, so a warp writes 32
// groups per 32 blocks and no unit is transformed twice (the shift kernel's
// split form transforms 2 virtual groups in 32 twice).
struct RotateParams {
  TransformParams t;
  uint4* gbase;       // out's 16-byte group
  char* out;          // element 0
  int64_t nw;         // output words: n es / 4
  int64_t h;          // output words of out's group before out
  int64_t r;          // word offset mod 4
  int64_t gofs;       // the group lane l completes is out's group + j + gofs (0 or -1)
  int64_t chunks;     // ceil(blocks / 32)
  uint64_t base_lo;   // block holding the stream's first word
  uint64_t base_hi;
  uint32_t s;         // the rotation kS, 1..3
  PhiloxRoundKeys rk;
};

// (lane - 1's last kS output words, this lane's first 4 - kS)
template <int kS>
__device__ __forceinline__ uint4 rotate_up(uint4 o) {
  const uint32_t n3 = __shfl_up_sync(0xFFFFFFFFu, o.w, 1);
  if constexpr (kS == 1) {
    return make_uint4(n3, o.x, o.y, o.z);
  } else {
    const uint32_t n2 = __shfl_up_sync(0xFFFFFFFFu, o.z, 1);
    if constexpr (kS == 2) {
      return make_uint4(n2, n3, o.x, o.y);
    } else {
      const uint32_t n1 = __shfl_up_sync(0xFFFFFFFFu, o.y, 1);
      return make_uint4(n1, n2, n3, o.x);
    }
  }
}

__device__ __forceinline__ uint32_t word_of(uint4 v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// Positions [q0, q1) of the 16-byte group at g, position q taking word
// q + kFrom of v; 8-byte elements go out whole (q0 and q1 even for them).
template <int V, int q0, int q1, int kFrom>
__device__ __forceinline__ void store_positions(uint4* g, uint4 v) {
  if constexpr (VInfo<V>::es == 4) {
#pragma unroll
    for (int q = q0; q < q1; ++q) reinterpret_cast<uint32_t*>(g)[q] = word_of(v, q + kFrom);
  } else {
#pragma unroll
    for (int q = q0; q < q1; q += 2)
      reinterpret_cast<uint2*>(g)[q >> 1] = make_uint2(word_of(v, q + kFrom), word_of(v, q + kFrom + 1));
  }
}

// The same with each output word checked against [0, nw) (edge chunks).
template <int V, int q0, int q1, int kFrom>
__device__ __forceinline__ void store_positions_checked(const RotateParams& p, int64_t G, uint4 v) {
  constexpr int kStep = VInfo<V>::es / 4;
#pragma unroll
  for (int q = q0; q < q1; q += kStep) {
    const int64_t i = 4 * G + q - p.h;
    if (i >= 0 && i < p.nw) {
      if constexpr (kStep == 1) {
        reinterpret_cast<uint32_t*>(p.out)[i] = word_of(v, q + kFrom);
      } else {
        reinterpret_cast<uint2*>(p.out)[i >> 1] =
            make_uint2(word_of(v, q + kFrom), word_of(v, q + kFrom + 1));
      }
    }
  }
}

template <int V, int U, bool kHiUniform, int kS>
__device__ __forceinline__ void philox_rotate_body(const RotateParams& p) {
  const int lane = threadIdx.x & 31;
  const int64_t TW = (int64_t)gridDim.x * (kThreads / 32);
  const int64_t c0 = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  // lane l of chunk c holds block j = 32 c + l; j, the counter and the group
  // address advance by increments (dj from chunk c to c + TW)
  const int64_t dj = TW * 32;
  int64_t j = c0 * 32 + lane;
  uint64_t lo = p.base_lo + (uint64_t)j;
  uint4* dst = p.gbase + (j + p.gofs);
  // the loop bound depends only on the warp: every shuffle has all 32 lanes
  for (int64_t c = c0; c < p.chunks;
       c += U * TW, j += U * dj, lo += (uint64_t)(U * dj), dst += U * dj) {
    uint4 b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t l = lo + (uint64_t)(u * dj);
      const uint64_t hh = kHiUniform ? p.base_hi : p.base_hi + ((l < p.base_lo) ? 1u : 0u);
      b[u] = philox4x32_10(ctr_from(l, hh), p.rk);
    }
    // every output word of this iteration's chunks lies inside the output
    // (uniform): words 128 c - r .. 128 c' + 127 - r, c' the last chunk
    const bool interior = c * 128 - p.r >= 0 && (c + (U - 1) * TW) * 128 + 127 - p.r < p.nw;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint4 o = block_outputs<V>(b[u], p.t);
      const uint4 g = rotate_up<kS>(o);
      if (interior) {
        uint4* gp = dst + u * dj;
        if (lane > 0) {
          *gp = g;
        } else {
          store_positions<V, kS, 4, 0>(gp, g);
        }
        if (lane == 31) store_positions<V, 0, kS, 4 - kS>(gp + 1, o);
      } else {
        const int64_t G = j + u * dj + p.gofs;
        if (lane > 0) {
          store_positions_checked<V, 0, 4, 0>(p, G, g);
        } else {
          store_positions_checked<V, kS, 4, 0>(p, G, g);
        }
        if (lane == 31) store_positions_checked<V, 0, kS, 4 - kS>(p, G + 1, o);
      }
    }
  }
}

// The rotation is the same for the whole grid: one loop per rotation, each
// with it a constant (8-byte elements rotate by one element only).
template <int V, int U, bool kHiUniform>
__device__ __forceinline__ void philox_rotate_phases(const RotateParams& p) {
  if constexpr (VInfo<V>::es == 8) {
    philox_rotate_body<V, U, kHiUniform, 2>(p);
  } else {
    switch (p.s) {
      case 1: philox_rotate_body<V, U, kHiUniform, 1>(p); break;
      case 2: philox_rotate_body<V, U, kHiUniform, 2>(p); break;
      default: philox_rotate_body<V, U, kHiUniform, 3>(p); break;
    }
  }
}

template <int V, int U, bool kHiUniform>
__global__ void __launch_bounds__(kThreads) philox_rotate_kernel(const __grid_constant__ RotateParams p) {
  philox_rotate_phases<V, U, kHiUniform>(p);
}

template <int V, int U, bool kHiUniform>
__global__ void __launch_bounds__(kThreads, 5) philox_rotate_kernel_5(const __grid_constant__ RotateParams p) {
  philox_rotate_phases<V, U, kHiUniform>(p);
}

// ------------------------------------------------------------ substreams
// num_streams streams whose every group is full (16-byte aligned streams of
// whole groups); stream s, group j is block base + s * sb + j.
struct MultiParams {
  TransformParams t;
  uint4* out;
  int64_t groups;     // groups per stream
  int64_t total;      // groups * num_streams
  uint64_t base_lo, base_hi;
  uint64_t sb_lo, sb_hi;      // block-counter stride between streams
  int64_t tq, tr;             // grid stride = tq * groups + tr
  uint64_t tqsb_lo, tqsb_hi;  // tq * sb
  PhiloxRoundKeys rk;
};

template <int V>
__global__ void __launch_bounds__(kThreads) philox_multi_kernel(const __grid_constant__ MultiParams p) {
  const int64_t T = (int64_t)gridDim.x * kThreads;
  int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (idx >= p.total) return;
  int64_t s = idx / p.groups;
  int64_t j = idx - s * p.groups;
  uint64_t sb_lo = p.base_lo, sb_hi = p.base_hi;  // block counter of group 0 of stream s
  {
    const uint64_t us = (uint64_t)s;
    add128(sb_lo, sb_hi, us * p.sb_lo, __umul64hi(us, p.sb_lo) + us * p.sb_hi);
  }
  for (; idx < p.total; idx += T) {
    uint64_t c_lo = sb_lo, c_hi = sb_hi;
    add128(c_lo, c_hi, (uint64_t)j, 0);
    p.out[idx] = block_outputs<V>(philox4x32_10(ctr_from(c_lo, c_hi), p.rk), p.t);
    j += p.tr;
    add128(sb_lo, sb_hi, p.tqsb_lo, p.tqsb_hi);
    if (j >= p.groups) {
      j -= p.groups;
      add128(sb_lo, sb_hi, p.sb_lo, p.sb_hi);
    }
  }
}

// Substreams at any word phase and pointer alignment: stream s writes
// out + s n elements from word offset off + s stride, and its 16-byte groups
// are found as in the shift kernel, per stream.  A warp takes one chunk of
// 30 groups of one stream, so the stream's phase, head and pair split are
// uniform across the warp: lanes compute 32 consecutive blocks, take the
// next block's first words from lane + 1, and, when the stream's start
// splits a Box-Muller pair, transform pair-aligned virtual groups one
// element earlier and exchange the straddling element (as kSplit above).
struct MultiShiftParams {
  TransformParams t;
  char* out;                 // element 0 of stream 0
  int64_t n;                 // elements per stream
  int64_t cps;               // warp chunks per stream
  int64_t total;             // cps * num_streams
  uint64_t off_lo, off_hi;   // word offset of stream 0
  uint64_t stride_lo, stride_hi;
  PhiloxRoundKeys rk;
};

constexpr int kMultiShiftPer = 30;

// Where stream s's (virtual) groups start, per stream of a multi-shift fill.
struct ShiftStream {
  char* sbase;      // element 0 of the stream
  uint4* gbase;     // its 16-byte aligned group 0
  int64_t head;     // elements of group 0 before sbase
  int64_t groups, jf, jl;
  uint64_t b_lo, b_hi;  // block of the first word of (virtual) group 0
  uint32_t ph;
  bool split;
};

template <int V>
__device__ __forceinline__ ShiftStream shift_stream(const MultiShiftParams& p, int64_t s) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  constexpr uint32_t kWpe = (uint32_t)(I::es / 4);  // words per element
  ShiftStream t;
  t.sbase = p.out + s * p.n * I::es;
  t.head = (int64_t)(((uintptr_t)t.sbase & 15u) / (uint32_t)I::es);
  t.gbase = reinterpret_cast<uint4*>((uintptr_t)t.sbase & ~(uintptr_t)15);
  t.split = I::epu == 2 && (t.head & 1) != 0;
  // first word of (virtual) group 0: off + s stride - head es/4 (one element
  // earlier when split), 128-bit
  uint64_t a_lo = p.off_lo, a_hi = p.off_hi;
  const uint64_t us = (uint64_t)s;
  add128(a_lo, a_hi, us * p.stride_lo, __umul64hi(us, p.stride_lo) + us * p.stride_hi);
  const uint64_t back = (uint64_t)t.head * kWpe + (t.split ? kWpe : 0u);
  a_hi -= (a_lo < back) ? 1u : 0u;
  a_lo -= back;
  t.b_lo = (a_lo >> 2) | (a_hi << 62);
  t.b_hi = a_hi >> 2;
  t.ph = (uint32_t)a_lo & 3u;
  t.groups = (t.head + p.n + kEpg - 1) / kEpg;
  t.jf = t.head > 0 ? 1 : 0;
  t.jl = ((t.head + p.n) % kEpg) != 0 ? t.groups - 1 : t.groups;
  return t;
}

template <int V>
__global__ void __launch_bounds__(kThreads) philox_multishift_kernel(
    const __grid_constant__ MultiShiftParams p) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  constexpr int kPer = kMultiShiftPer;
  const int lane = threadIdx.x & 31;
  // each warp takes a run of consecutive chunks (chunk c = stream c / cps,
  // chunk c mod cps of it), so a stream's set-up is redone only when the run
  // enters the next stream; the loop bound depends only on the warp
  const int64_t W = (int64_t)gridDim.x * (kThreads / 32);
  const int64_t w = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const int64_t L = (p.total + W - 1) / W;
  int64_t c = w * L;
  const int64_t c_end = (c + L) < p.total ? (c + L) : p.total;
  if (c >= c_end) return;
  int64_t s = c / p.cps;
  int64_t k = c - s * p.cps;
  ShiftStream t = shift_stream<V>(p, s);
  for (; c < c_end; ++c) {
    const int64_t j = k * kPer + lane;
    const uint64_t c_lo = t.b_lo + (uint64_t)j;
    const uint64_t c_hi = t.b_hi + ((c_lo < t.b_lo) ? 1u : 0u);
    const uint4 b = philox4x32_10(ctr_from(c_lo, c_hi), p.rk);
    // the stream's phase and split are the same for the whole warp, so the
    // exchanges run on all 32 lanes or on none: a stream at phase 0 skips the
    // word exchange (16384 x 65537 at a stride of 2^40 + 1, half the streams
    // at phase 0: bits 1.108 -> 1.030 ms, FP32 uniform 1.219 -> 1.145 ms)
    uint4 w = b;
    if (t.ph != 0) w = shift_words(b, t.ph);
    uint4 o = block_outputs<V>(w, p.t);
    if constexpr (I::epu == 2) {
      if (t.split) o = split_group<V>(o);
    }
    if (k * kPer >= t.jf && k * kPer + kPer <= t.jl) {  // whole groups (uniform)
      if (lane < kPer) t.gbase[j] = o;
    } else if (lane < kPer && j < t.groups) {
      const int64_t e0 = j * kEpg - t.head;
      if (e0 >= 0 && e0 + kEpg <= p.n) {
        t.gbase[j] = o;
      } else {
        store_partial<V>(t.sbase, e0, p.n, o);
      }
    }
    if (++k == p.cps) {
      k = 0;
      ++s;
      if (c + 1 < c_end) t = shift_stream<V>(p, s);
    }
  }
}

// CTAs per SM a launch may use, from the tuned geometry: 1..16 a cap on the
// resident CTAs; 17 and above (geom - 16) waves of resident CTAs, each CTA
// taking that fraction of a resident CTA's share of the grid-stride loop, so
// that the hardware refills an SM as its CTAs finish instead of the SM
// emptying out as the faster warps of long-lived CTAs finish first (ncu: a
// single persistent wave kept 33 of 48 possible warps active); 0, the
// built-in choice, is 8 waves (within 1 % of the best wave count for every
// fill at n = 10^9; one wave was up to 6 % slower).
int ctas_cap(int occ, int32_t geom) {
  if (geom == 0) return occ * 8;
  if (geom > 16) return occ * (geom - 16);
  return geom < occ ? (int)geom : occ;
}

template <typename K>
int blocks_per_sm(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0) != cudaSuccess ||
      b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}

// Launches the shift kernel: words of (virtual) group 0 start at word a of
// the stream (128-bit, a = off - head words, one element earlier for kSplit).
template <int V, bool kSplit>
void launch_shift(ShiftParams& p, uint64_t a_lo, uint64_t a_hi, int sms, int32_t geom,
                  cudaStream_t stream) {
  constexpr int kPer = shift_per_warp<kSplit>();
  constexpr int kU = blocks_per_thread<V>();
  p.base_lo = (a_lo >> 2) | (a_hi << 62);
  p.base_hi = a_hi >> 2;
  p.ph = (uint32_t)(a_lo & 3u);
  p.chunks = (p.groups + kPer - 1) / kPer;
  void (*k_uni)(const ShiftParams);
  void (*k_carry)(const ShiftParams);
  if constexpr (stream_wants_5_ctas<V>()) {
    k_uni = philox_shift_kernel_5<V, kU, true, kSplit>;
    k_carry = philox_shift_kernel_5<V, kU, false, kSplit>;
  } else {
    k_uni = philox_shift_kernel<V, kU, true, kSplit>;
    k_carry = philox_shift_kernel<V, kU, false, kSplit>;
  }
  static std::atomic<int> occ[2] = {{0}, {0}};
  int o = occ[0].load(std::memory_order_relaxed);
  if (o == 0) {
    o = blocks_per_sm(k_uni);
    occ[0].store(o, std::memory_order_relaxed);
    occ[1].store(blocks_per_sm(k_carry), std::memory_order_relaxed);
  }
  const int64_t warps = (p.chunks + kU - 1) / kU;
  int64_t grid = (warps + (kThreads / 32) - 1) / (kThreads / 32);
  if (grid < 1) grid = 1;
  const int64_t cap = (int64_t)sms * ctas_cap(o, geom);
  if (grid > cap) grid = cap;
  // blocks touched: below (chunks + kU * warps in flight) * kPer + 32 past base
  const uint64_t reach =
      (uint64_t)(p.chunks + (int64_t)kU * grid * (kThreads / 32) + 1) * (uint64_t)kPer + 64u;
  const bool hi_uniform = p.base_lo + reach >= p.base_lo;
  if (!hi_uniform) {
    const int64_t cap2 = (int64_t)sms * ctas_cap(occ[1].load(std::memory_order_relaxed), geom);
    if (grid > cap2) grid = cap2;
  }
  (hi_uniform ? k_uni : k_carry)<<<(unsigned)grid, kThreads, 0, stream>>>(p);
}

// Launches the rotate kernel (units inside blocks, output start at another
// phase); p.t, p.out, p.gbase, p.nw, p.h, p.rk are set by the caller.
template <int V>
void launch_rotate(RotateParams& p, uint64_t off_lo, uint64_t off_hi, int sms, int32_t geom,
                   cudaStream_t stream) {
  constexpr int kU = blocks_per_thread<V>();
  p.r = (int64_t)(off_lo & 3u);
  const int64_t d = p.h - p.r;
  p.s = (uint32_t)((d + 4) & 3);
  p.gofs = d < 0 ? -1 : 0;
  p.base_lo = (off_lo >> 2) | (off_hi << 62);
  p.base_hi = off_hi >> 2;
  const int64_t blocks = (p.nw - 1 + p.r) / 4 + 1;
  p.chunks = (blocks + 31) / 32;
  void (*k_uni)(const RotateParams);
  void (*k_carry)(const RotateParams);
  // the FP64 Box-Muller variants gain from a fifth CTA as in the stream
  // kernel; the FP32 ones would spill under its register cap here
  if constexpr (stream_wants_5_ctas<V>() && VInfo<V>::es == 8) {
    k_uni = philox_rotate_kernel_5<V, kU, true>;
    k_carry = philox_rotate_kernel_5<V, kU, false>;
  } else {
    k_uni = philox_rotate_kernel<V, kU, true>;
    k_carry = philox_rotate_kernel<V, kU, false>;
  }
  static std::atomic<int> occ[2] = {{0}, {0}};
  int o = occ[0].load(std::memory_order_relaxed);
  if (o == 0) {
    o = blocks_per_sm(k_uni);
    occ[0].store(o, std::memory_order_relaxed);
    occ[1].store(blocks_per_sm(k_carry), std::memory_order_relaxed);
  }
  const int64_t warps = (p.chunks + kU - 1) / kU;
  int64_t grid = (warps + (kThreads / 32) - 1) / (kThreads / 32);
  if (grid < 1) grid = 1;
  const int64_t cap = (int64_t)sms * ctas_cap(o, geom);
  if (grid > cap) grid = cap;
  // blocks touched: below (chunks + kU * warps in flight) * 32 past base
  const uint64_t reach = (uint64_t)(p.chunks + (int64_t)kU * grid * (kThreads / 32) + 1) * 32u;
  const bool hi_uniform = p.base_lo + reach >= p.base_lo;
  if (!hi_uniform) {
    const int64_t cap2 = (int64_t)sms * ctas_cap(occ[1].load(std::memory_order_relaxed), geom);
    if (grid > cap2) grid = cap2;
  }
  (hi_uniform ? k_uni : k_carry)<<<(unsigned)grid, kThreads, 0, stream>>>(p);
}

template <int V>
grng_status launch_variant(const FillRequest& r, cudaStream_t stream) {
  using I = VInfo<V>;
  constexpr int kEpg = 16 / I::es;
  int dev = 0;
  const int sms = current_device_sms(&dev);
  const int32_t geom = fill_geometry(GRNG_PHILOX4X32X10, V, r.n * r.num_streams);
  const uintptr_t addr = (uintptr_t)r.out;
  const uint32_t phase_w = (uint32_t)((addr & 15u) / 4u);  // output words before out in group 0
  const uint64_t stream_bytes = (uint64_t)r.n * I::es;
  // same alignment phase for every stream, and a block-multiple stride
  const bool uniform_streams =
      r.num_streams == 1 || ((stream_bytes % 16u) == 0 && (r.stride_lo & 3u) == 0);
  const bool fast = uniform_streams && ((r.off_lo - phase_w) & 3u) == 0 &&
                    (phase_w % (uint32_t)I::wpu) == 0;

  // base block counter = (off - phase_w) / 4 with a 128-bit borrow
  const uint64_t lo0 = r.off_lo - phase_w;
  const uint64_t hi0 = r.off_hi - ((r.off_lo < phase_w) ? 1u : 0u);
  const uint64_t base_lo = (lo0 >> 2) | (hi0 << 62);
  const uint64_t base_hi = hi0 >> 2;
  const int64_t head = (int64_t)(phase_w * 4u / I::es);
  const int64_t groups = (head + r.n + kEpg - 1) / kEpg;
  if (fast && r.num_streams == 1) {
    StreamParams p;
    p.t = r.t;
    p.out = r.out;
    p.gbase = reinterpret_cast<uint4*>(addr - phase_w * 4u);
    p.n = r.n;
    p.head = head;
    p.base_lo = base_lo;
    p.base_hi = base_hi;
    p.rk = philox_round_keys(r.key[0], r.key[1]);
    // full groups: the first group is partial when head > 0, the last one
    // when the end is not on a group boundary (or both are the same group)
    int64_t jf = head > 0 ? 1 : 0;
    int64_t jl = ((head + r.n) % kEpg) != 0 ? groups - 1 : groups;
    p.edge[0] = p.edge[1] = -1;
    if (jf > jl) {  // a single partial group
      p.edge[0] = 0;
      jf = jl = 0;
    } else {
      if (head > 0) p.edge[0] = 0;
      if (jl < groups) p.edge[1] = groups - 1;
    }
    p.jf = jf;
    p.jl = jl;
    constexpr int kU = blocks_per_thread<V>();
    const bool hi_uniform = base_lo + (uint64_t)groups >= base_lo;  // no carry into the top half
    void (*kernel)(const StreamParams);
    if constexpr (stream_wants_5_ctas<V>()) {
      kernel = hi_uniform ? philox_stream_kernel_5<V, kU, true> : philox_stream_kernel_5<V, kU, false>;
    } else {
      kernel = hi_uniform ? philox_stream_kernel<V, kU, true> : philox_stream_kernel<V, kU, false>;
    }
    // resident CTAs per SM, found once per kernel (atomic: launches may come
    // from several host threads)
    static std::atomic<int> occ[2] = {{0}, {0}};
    int o = occ[hi_uniform ? 1 : 0].load(std::memory_order_relaxed);
    if (o == 0) {
      o = blocks_per_sm(kernel);
      occ[hi_uniform ? 1 : 0].store(o, std::memory_order_relaxed);
    }
    const int64_t work = (jl - jf + (int64_t)kU - 1) / kU;
    int64_t grid = (work + kThreads - 1) / kThreads;
    if (grid < 1) grid = 1;
    const int64_t cap = (int64_t)sms * ctas_cap(o, geom);
    if (grid > cap) grid = cap;
    kernel<<<(unsigned)grid, kThreads, 0, stream>>>(p);
  } else if (fast && head == 0 && (stream_bytes % 16u) == 0) {
    MultiParams p;
    p.t = r.t;
    p.out = reinterpret_cast<uint4*>(r.out);
    p.groups = groups;
    p.total = groups * r.num_streams;
    p.base_lo = base_lo;
    p.base_hi = base_hi;
    p.sb_lo = (r.stride_lo >> 2) | (r.stride_hi << 62);
    p.sb_hi = r.stride_hi >> 2;
    p.rk = philox_round_keys(r.key[0], r.key[1]);
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ == 0) {
      occ = blocks_per_sm(philox_multi_kernel<V>);
      occ_cache.store(occ, std::memory_order_relaxed);
    }
    int64_t grid = (p.total + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sms * ctas_cap(occ, geom);
    if (grid > cap) grid = cap;
    const int64_t gstride = grid * kThreads;
    p.tq = gstride / p.groups;
    p.tr = gstride - p.tq * p.groups;
    const unsigned __int128 tqsb =
        (unsigned __int128)(uint64_t)p.tq *
        (((unsigned __int128)p.sb_hi << 64) | (unsigned __int128)p.sb_lo);
    p.tqsb_lo = (uint64_t)tqsb;
    p.tqsb_hi = (uint64_t)(tqsb >> 64);
    philox_multi_kernel<V><<<(unsigned)grid, kThreads, 0, stream>>>(p);
  } else if (I::wpu >= 2 && r.num_streams == 1 && (r.off_lo % (uint64_t)I::wpu) == 0) {
    // one stream whose units lie inside counter blocks, the output start at
    // another phase (e.g. a Box-Muller pair split by the pointer)
    if constexpr (I::wpu >= 2) {
      RotateParams p;
      p.t = r.t;
      p.out = reinterpret_cast<char*>(r.out);
      p.gbase = reinterpret_cast<uint4*>(addr - phase_w * 4u);
      p.nw = r.n * (I::es / 4);
      p.h = (int64_t)phase_w;
      p.rk = philox_round_keys(r.key[0], r.key[1]);
      launch_rotate<V>(p, r.off_lo, r.off_hi, sms, geom, stream);
    }
  } else if (r.num_streams == 1 &&
             ((phase_w % (uint32_t)I::wpu) == 0 || (I::epu == 2 && (head & 1) != 0))) {
    // one stream at another word phase, or a pair split by the output's start
    ShiftParams p;
    p.t = r.t;
    p.out = r.out;
    p.gbase = reinterpret_cast<uint4*>(addr - phase_w * 4u);
    p.n = r.n;
    p.head = head;
    p.groups = groups;
    p.jf = head > 0 ? 1 : 0;
    p.jl = ((head + r.n) % kEpg) != 0 ? groups - 1 : groups;
    p.rk = philox_round_keys(r.key[0], r.key[1]);
    if ((phase_w % (uint32_t)I::wpu) == 0) {
      launch_shift<V, false>(p, lo0, hi0, sms, geom, stream);
    } else if constexpr (I::epu == 2) {
      // the virtual groups start one element (es / 4 words) earlier
      const uint32_t pv = phase_w + (uint32_t)(I::es / 4);
      const uint64_t a_lo = r.off_lo - pv;
      const uint64_t a_hi = r.off_hi - ((r.off_lo < pv) ? 1u : 0u);
      launch_shift<V, true>(p, a_lo, a_hi, sms, geom, stream);
    }
  } else {
    // substreams at any other phase or alignment
    MultiShiftParams p;
    p.t = r.t;
    p.out = reinterpret_cast<char*>(r.out);
    p.n = r.n;
    // groups of a stream with the largest head (16 / es - 1 elements)
    const int64_t max_groups = (r.n + (kEpg - 1) + kEpg - 1) / kEpg;
    p.cps = (max_groups + kMultiShiftPer - 1) / kMultiShiftPer;
    p.total = p.cps * r.num_streams;
    p.off_lo = r.off_lo;
    p.off_hi = r.off_hi;
    p.stride_lo = r.stride_lo;
    p.stride_hi = r.stride_hi;
    p.rk = philox_round_keys(r.key[0], r.key[1]);
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ == 0) {
      occ = blocks_per_sm(philox_multishift_kernel<V>);
      occ_cache.store(occ, std::memory_order_relaxed);
    }
    int64_t grid = (p.total + (kThreads / 32) - 1) / (kThreads / 32);
    const int64_t cap = (int64_t)sms * ctas_cap(occ, geom);
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    philox_multishift_kernel<V><<<(unsigned)grid, kThreads, 0, stream>>>(p);
  }
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error("Philox fill launch failed: %s", cudaGetErrorString(err));
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}

}  // namespace

grng_status launch_philox(const FillRequest& r, CUstream_st* stream) {
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
