// Internal types shared by the host C ABI (capi.cpp) and the kernel launchers
// (philox_kernels.cu, mrg_kernels.cu).  Not part of the public interface.
#pragma once

#include <cstdint>

#include "grng.h"

struct CUstream_st;

namespace grng {

// One variant per (distribution, dtype) plus exact fast forms of the uniform
// transform that give bit-identical results (see TransformParams).
enum Variant : int {
  V_BITS = 0,      // uint32 words
  V_U01_F32 = 1,   // uniform F32 on [0, 1): u itself (0 + 1 * u == u exactly)
  V_UNI_F32 = 2,   // uniform F32 on [a, b): RN mul, RN add, clamp below b
  V_U01_F64 = 3,   // uniform F64 on [0, 1)
  V_AFF_F64 = 4,   // uniform F64 on [a, b) when a + (b - a) u is exact: integer form
  V_UNI_F64 = 5,   // uniform F64 on [a, b): FP64 RN mul, RN add, clamp
  V_GAUSS_F32 = 6,
  V_LOGN_F32 = 7,
  V_GAUSS_F64 = 8,
  V_LOGN_F64 = 9,
  V_ICDF_GAUSS_F32 = 10,  // inverse-CDF gaussian / lognormal: one uniform per output
  V_ICDF_LOGN_F32 = 11,
  V_ICDF_GAUSS_F64 = 12,
  V_ICDF_LOGN_F64 = 13,
  V_STDGAUSS_F64 = 14,  // F64 gaussian with (0, 1): no FP64 affine step at all
  V_COUNT = 15
};

// Geometry of a variant.  Every variant produces 4 output bytes per word it
// consumes, so a 16-byte output group always corresponds to 4 words.
struct VariantInfo {
  int es;   // element size in bytes
  int wpu;  // words per unit (a unit is one output, or one Box-Muller pair)
  int epu;  // elements per unit
};

inline VariantInfo variant_info(int v) {
  switch (v) {
    case V_BITS: case V_U01_F32: case V_UNI_F32: return {4, 1, 1};
    case V_U01_F64: case V_AFF_F64: case V_UNI_F64: return {8, 2, 1};
    case V_GAUSS_F32: case V_LOGN_F32: return {4, 2, 2};
    case V_ICDF_GAUSS_F32: case V_ICDF_LOGN_F32: return {4, 1, 1};
    case V_ICDF_GAUSS_F64: case V_ICDF_LOGN_F64: return {8, 2, 1};
    default: return {8, 4, 2};  // V_GAUSS_F64, V_LOGN_F64, V_STDGAUSS_F64
  }
}

// Distribution parameters as the kernels use them.
struct TransformParams {
  float fa, fd, fb, fbprev;   // F32 uniform: a, b - a, b, largest float below b
  float fmean, fsd;           // F32 gaussian (mean, sd) / lognormal (m, s)
  double da, dd, db, dbprev;  // F64 uniform
  // F64 uniform on [a, b) with the product d u in integers: d = (rd_hi 2^32 +
  // rd_lo) 2^rd_exp, its 53-bit significand; r_int = 0 keeps the FP64
  // product; r_xthr = the smallest 53-bit x whose a + d x 2^-53 (two
  // roundings) reaches b, 2^53 if none
  uint32_t rd_hi, rd_lo;
  int32_t rd_exp, r_int;
  uint64_t r_xthr;
  double dmean, dsd;          // F64 gaussian / lognormal
  int64_t aff_a;              // F64 exact affine: r = (aff_a + x) 2^aff_exp, x = 53-bit word
  int32_t aff_exp;
  // F64 lognormal in fixed point: exp(m) = ln_em_mant 2^ln_em_exp, s = ln_s_mant 2^ln_s_exp;
  // ln_fast = 0 keeps every output on the FP64 path
  int32_t ln_fast;
  uint64_t ln_em_mant, ln_s_mant;
  int32_t ln_em_exp, ln_s_exp;
};

// One fill request as the launchers see it: num_streams streams of n
// elements; stream s starts at word offset off + s * stride and writes
// out + s * n elements.
struct FillRequest {
  int variant;
  int engine_kind;
  int64_t n;
  int64_t num_streams;
  uint64_t off_lo, off_hi;
  uint64_t stride_lo, stride_hi;
  void* out;
  TransformParams t;
  uint32_t key[2];     // Philox key
  uint32_t mrg[6];     // MRG32k3a state at word offset off: x1[3], x2[3]
};

// One request of a batched fill as the device sees it (batch.cu).
struct BatchReq {
  TransformParams t;
  uint64_t out;        // device address of element 0
  int64_t n;           // elements
  int64_t groups;      // 16-byte groups covering [out, out + n) (with the head)
  int64_t first_tile;
  uint64_t adv_lo, adv_hi;  // words the engine advances per launch
  uint32_t key0, key1;
  int32_t variant;
  int32_t head;        // elements of group 0 before out
};

// A Philox fill described for plan_parts: key, starting word offset,
// distribution (variant + parameters), size and device output address.
struct PartDesc {
  uint32_t key0, key1;
  uint64_t off_lo, off_hi;
  TransformParams t;
  int variant;
  int es;              // element size
  int64_t n;
  uint64_t out;
};

// Writes batch records, starting offsets and the tile -> part map for `count`
// parts (no per-launch advance); returns the number of tiles, or -1 when it
// would exceed tile_cap.
int64_t plan_parts(const PartDesc* parts, int32_t count, int ipt, BatchReq* reqs_out,
                   uint64_t* offs_out, int32_t* tiles_out, int64_t tile_cap);

// Enqueues the batched fill over device copies of those tables.
grng_status enqueue_fill(const BatchReq* d_reqs, const uint64_t* d_offs, const int32_t* d_tiles,
                         int64_t tiles, int ipt, int64_t grid, CUstream_st* stream);

// Kernel launchers; return GRNG_OK or GRNG_ERR_CUDA (detail via set_error).
grng_status launch_philox(const FillRequest& r, CUstream_st* stream);
grng_status launch_mrg(const FillRequest& r, CUstream_st* stream);
// Applies a variant to n outputs' worth of caller-supplied device words.
grng_status launch_transform(int variant, const TransformParams& t, const uint32_t* words,
                             int64_t n, void* out, CUstream_st* stream);

// Checks a distribution and fills the kernels' parameters and variant.
grng_status fill_transform_params(const grng_distribution* d, TransformParams* t, int* variant);

// Records an error message for grng_last_error() on this thread.
void set_error(const char* fmt, ...);

// Multiprocessor count of the current device (cached per device).
int current_device_sms(int* device_out);

// Tuned launch geometry of a fill of n elements (tune.cpp): Philox4x32-10,
// the cap on resident CTAs per SM; MRG32k3a, threads per SM of the chunk
// plan in units of 256; 0 = the launcher's built-in choice.
int32_t fill_geometry(int engine_kind, int variant, int64_t n);

}  // namespace grng
