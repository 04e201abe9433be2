// FP64 inverse CDF of the standard normal in fixed-point integer arithmetic.
//
// For p in (0, 1/2], t = -Phi^-1(p) is computed as a function of
// w = sqrt(-2 ln p): -ln p and the square root come from the fixed-point
// Box-Muller code (bm64_fixed.cuh), and t(w) from a piecewise degree-8
// polynomial (icdf64_tables.h, written by gen_icdf64_tables.py: 46 segments
// of D = w - w0, w0 = sqrt(2 ln 2), fit errors below 1e-17 of max(1, t)).
// Horner's rule runs in 2^-59 units; the two top steps, whose terms are
// below 2^-24, use 32-bit products.  No FP64 instruction is involved, so
// the narrow FP64 pipe of this part does not bound it.
#pragma once

#include <cstdint>

#include "bm64_fixed.cuh"
#include "icdf64_tables.h"

namespace grng {
namespace icdf64 {

#if defined(__CUDACC__)
__device__ const int64_t d_coef[GRNG_ICDF64_SEGS * (GRNG_ICDF64_DEG + 1)] = GRNG_ICDF64_COEF;
#endif
static const int64_t h_coef[GRNG_ICDF64_SEGS * (GRNG_ICDF64_DEG + 1)] = GRNG_ICDF64_COEF;

GRNG_BM_HD int64_t coef(uint32_t i) {
#if defined(__CUDA_ARCH__)
  return __ldg(&d_coef[i]);
#else
  return h_coef[i];
#endif
}

// floor(a s 2^-64) for signed a and s in [0, 2^64), at most 2 below: the
// unsigned high product of a's two's-complement pattern exceeds it by s when
// a < 0.
GRNG_BM_HD int64_t mulhi_su(int64_t a, uint64_t s) {
  return (int64_t)(bm64::umulhi_apx((uint64_t)a, s) - (a < 0 ? s : 0ull));
}

// t 2^59 with t = -Phi^-1(p), p = m1 2^-53, m1 in [1, 2^52] (p <= 1/2).
GRNG_BM_HD uint64_t neg_icdf(uint64_t m1) {
  uint64_t lm, sq;
  int le, se;
  bm64::neg_log(m1, lm, le);                 // -ln p = lm 2^le
  bm64::sqrt2x(lm, le, sq, se);              // w = sqrt(-2 ln p) = sq 2^se
  const int sh = se + 60;                    // w 2^60 = sq 2^sh, sh in -1..2
  const uint64_t W60 = sh >= 0 ? (sq << sh) : (sq >> (-sh));
  const uint64_t D = W60 > kW0_60 ? W60 - kW0_60 : 0ull;  // (w - w0) 2^60
  // segment j and the position S = s 2^64 inside it
  uint32_t j;
  uint64_t S;
  if (D < (3ull << 58)) {                    // D < 3/4: width 1/16
    j = (uint32_t)(D >> 56);
    S = (D & ((1ull << 56) - 1)) << 8;
  } else if (D < (5ull << 59)) {             // D < 5/2: width 1/8
    const uint64_t E = D - (3ull << 58);
    j = 12u + (uint32_t)(E >> 57);
    S = (E & ((1ull << 57) - 1)) << 7;
  } else {                                   // width 1/4
    const uint64_t E = D - (5ull << 59);
    j = 26u + (uint32_t)(E >> 58);
    S = (E & ((1ull << 58) - 1)) << 6;
    if (j >= GRNG_ICDF64_SEGS) {             // only past p = 2^-53
      j = GRNG_ICDF64_SEGS - 1;
      S = ~0ull;
    }
  }
  const uint32_t base = j * (GRNG_ICDF64_DEG + 1);
  const int32_t s31 = (int32_t)(S >> 33);    // s 2^31
  // |c8| < 2^24.1, |c7| < 2^28.6, |c6| < 2^32.7 (units 2^-59)
  const int32_t b7 = (int32_t)coef(base + 7) +
                     (int32_t)(((int64_t)(int32_t)coef(base + 8) * s31) >> 31);
  int64_t b = coef(base + 6) + (((int64_t)b7 * s31) >> 31);
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int i = 5; i >= 0; --i) b = coef(base + i) + mulhi_su(b, S);
  return b > 0 ? (uint64_t)b : 0ull;
}

// z = Phi^-1(u) for u = (x + 1/2) 2^-52, x 52-bit: t 2^59 and the sign.
GRNG_BM_HD uint64_t icdf_t59(uint64_t x, bool& negative) {
  negative = x < (1ull << 51);               // u < 1/2
  const uint64_t m1 = negative ? 2 * x + 1 : (1ull << 53) - 2 * x - 1;
  return neg_icdf(m1);
}

}  // namespace icdf64
}  // namespace grng
