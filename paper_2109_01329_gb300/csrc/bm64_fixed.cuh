// FP64 Box-Muller in 64-bit fixed-point integer arithmetic.
//
// The double-precision pipe of this part is narrow (a Box-Muller pair in FP64
// math takes ~60x longer than the same pair's HBM time), so the FP64
// gaussian is computed with 32x32 -> 64-bit integer multiplies instead, and
// only the final result is assembled into an IEEE double (round to nearest).
//
//   z0 = rho cos(2 pi u2), z1 = rho sin(2 pi u2), rho = sqrt(-2 ln u1),
//   u1 = (x1 + 1) 2^-53 in (0, 1], u2 = x2 2^-53 in [0, 1), x1, x2 53-bit.
//
// -ln u1:  u1 = 2^-e (1 - delta) with e >= 0, delta in (0, 1/2]; a table
//          factor c_i ~ 1/(1 - i/1024) reduces it to -ln(1 - delta) =
//          ln c_i - ln(1 - r), 0 <= r < 2^-9, whose series r + r^2/2 + ... +
//          r^7/7 is summed by Horner (inner terms in 32-bit fixed point).  For i = 0 (u1 within 2^-10 of 1),
//          r = delta exactly, so -ln u1 keeps full relative accuracy even
//          for the smallest delta, 2^-53.
// rho:     1 / sqrt by two Newton steps from the FP32 reciprocal square root
//          (the first one on the 24-bit seed with narrow products), then
//          sqrt = x / sqrt(x).
// sincos:  octant symmetry, a 1025-entry table of sin / cos at multiples of
//          2 pi / 8192 and two-term series for the residual angle
//          phi < 2 pi 2^-13.
// Error: below 2^-55 relative on rho and 2^-60 absolute on sin and cos
// before the final rounding to double.
#pragma once

#include <cstdint>

#include "bm64_tables.h"

#if defined(__CUDACC__)
#define GRNG_BM_HD __host__ __device__ __forceinline__
#else
#define GRNG_BM_HD inline
#endif

namespace grng {
namespace bm64 {

#if defined(__CUDACC__)
__device__ const uint32_t d_logc[GRNG_BM64_LOGC_LEN] = GRNG_BM64_LOGC;
__device__ const uint64_t d_logt[GRNG_BM64_LOGT_LEN] = GRNG_BM64_LOGT;
__device__ const uint64_t d_sint[GRNG_BM64_SINT_LEN] = GRNG_BM64_SINT;
__device__ const uint64_t d_cost[GRNG_BM64_COST_LEN] = GRNG_BM64_COST;
#endif
static const uint32_t h_logc[GRNG_BM64_LOGC_LEN] = GRNG_BM64_LOGC;
static const uint64_t h_logt[GRNG_BM64_LOGT_LEN] = GRNG_BM64_LOGT;
static const uint64_t h_sint[GRNG_BM64_SINT_LEN] = GRNG_BM64_SINT;
static const uint64_t h_cost[GRNG_BM64_COST_LEN] = GRNG_BM64_COST;

GRNG_BM_HD uint32_t logc(uint32_t i) {
#if defined(__CUDA_ARCH__)
  return __ldg(&d_logc[i]);
#else
  return h_logc[i];
#endif
}
GRNG_BM_HD uint64_t logt(uint32_t i) {
#if defined(__CUDA_ARCH__)
  return __ldg(&d_logt[i]);
#else
  return h_logt[i];
#endif
}
GRNG_BM_HD uint64_t sint(uint32_t j) {
#if defined(__CUDA_ARCH__)
  return __ldg(&d_sint[j]);
#else
  return h_sint[j];
#endif
}
GRNG_BM_HD uint64_t cost(uint32_t j) {
#if defined(__CUDA_ARCH__)
  return __ldg(&d_cost[j]);
#else
  return h_cost[j];
#endif
}

GRNG_BM_HD uint64_t umulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

// High 64 bits of a * b from three 32x32 -> 64-bit products: the low x low
// product and the carry out of the low halves of the two cross products are
// dropped, so the result is at most 2 below the exact high word (2 units of
// the 2^-64 scale used throughout).  Where two halves of one product are
// spliced together the exact form below is used instead.
GRNG_BM_HD uint64_t umulhi_apx(uint64_t a, uint64_t b) {
  const uint64_t ah = a >> 32, al = (uint32_t)a, bh = b >> 32, bl = (uint32_t)b;
  return ah * bh + ((ah * bl) >> 32) + ((al * bh) >> 32);
}

// Exact 96-bit product of a 64-bit and a 32-bit value: hi = (a c) >> 32,
// lo32 = (a c) mod 2^32.
GRNG_BM_HD void mul64x32(uint64_t a, uint32_t c, uint64_t& hi, uint32_t& lo32) {
  const uint64_t l = (a & 0xFFFFFFFFull) * c;
  hi = (a >> 32) * c + (l >> 32);
  lo32 = (uint32_t)l;
}

GRNG_BM_HD uint32_t __umulhi32(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a * b) >> 32);
}

GRNG_BM_HD int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

GRNG_BM_HD float rsqrt_seed(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / __builtin_sqrtf(x);
#endif
}

// -ln(u1) for u1 = m1 2^-53, m1 in [1, 2^53), as lm 2^le with lm normalised
// (top bit set).  m1 = 2^53 (u1 = 1) is handled by the caller.
GRNG_BM_HD void neg_log(uint64_t m1, uint64_t& lm, int& le) {
  const int q = 63 - clz64(m1);             // 0..52
  const uint64_t e = (uint64_t)(52 - q);    // u1 = 2^-e (1 - delta)
  const uint64_t M = m1 << (63 - q);        // (1 - delta) 2^64, top bit set
  const uint64_t D = 0ull - M;              // delta 2^64 in (0, 2^63]
  const uint32_t i = (uint32_t)(D >> 54);   // 0..512
  const uint32_t C = logc(i);               // c_i 2^24
  // r 2^64 = 2^64 - M C 2^-24 (truncating M C 2^-24 leaves r >= 0); the
  // 96-bit product M C is exact, and M C 2^-24 = (hi << 8) | (lo32 >> 24)
  uint64_t mc_hi;
  uint32_t mc_lo;
  mul64x32(M, C, mc_hi, mc_lo);
  const uint64_t R = 0ull - ((mc_hi << 8) | (uint64_t)(mc_lo >> 24));
  // -ln(1 - r) = r + r^2 (1/2 + r (1/3 + r B4)), B4 = 1/4 + r/5 + r^2/6 + r^3/7.
  // r < 2^-9, so r^4 B4 is below 2^-36: B4 in 32-bit fixed point (its error
  // enters S below 2^-67), the outer two Horner steps in 64-bit.
  const uint32_t r32 = (uint32_t)(R >> 32);             // r 2^32 < 2^23
  uint32_t b4 = kInv7_32;
  b4 = kInv6_32 + __umulhi32(r32, b4);
  b4 = kInv5_32 + __umulhi32(r32, b4);
  b4 = kInv4_32 + __umulhi32(r32, b4);
  uint64_t b4r_hi;                                       // (R b4) >> 32 = r B4 2^64
  uint32_t b4r_lo;
  mul64x32(R, b4, b4r_hi, b4r_lo);
  const uint64_t B3 = kInv3 + b4r_hi;
  const uint64_t B2 = kInv2 + umulhi_apx(R, B3);
  const uint64_t S = R + umulhi_apx(umulhi_apx(R, R), B2);
  // L 2^64 = e ln 2 + ln c_i + S, as a 128-bit sum (e ln 2 exactly: 64 x 32)
  uint64_t ln2e_hi;
  uint32_t ln2e_lo;
  mul64x32(kLn2, (uint32_t)e, ln2e_hi, ln2e_lo);
  uint64_t lo = (ln2e_hi << 32) | ln2e_lo;
  uint64_t hi = ln2e_hi >> 32;
  const uint64_t T = logt(i);
  lo += T;
  hi += (lo < T) ? 1u : 0u;
  lo += S;
  hi += (lo < S) ? 1u : 0u;
  if (hi != 0) {
    const int nz = clz64(hi);               // 58..63
    lm = (hi << nz) | (lo >> (64 - nz));
    le = -nz;
  } else {
    const int nz = clz64(lo);               // lo != 0 since u1 < 1
    lm = lo << nz;
    le = -64 - nz;
  }
}

// sqrt(2 lm 2^le) as sq 2^se, sq in [2^61, 2^62].
GRNG_BM_HD void sqrt2x(uint64_t lm, int le, uint64_t& sq, int& se) {
  int E = le + 1;                           // 2L = lm 2^E
  uint64_t X = lm;
  if (E & 1) {                              // make the exponent even
    X = lm >> 1;
    E += 1;
  }
  // x = X 2^-64 in [1/4, 1); y = 1/sqrt(x) in (1, 2] kept as Y = y 2^62
  const float xf = (float)(uint32_t)(X >> 40) * 0x1p-24f;
  const float yf = rsqrt_seed(xf);
  uint32_t yb;
  __builtin_memcpy(&yb, &yf, 4);
  const int ey = (int)((yb >> 23) & 0xFFu) - 127;   // 0 or 1
  // first Newton step from the 24-bit seed y0 = m24 2^(ey - 23): its square
  // and its product with (3 - x y0^2) need only 24 x 32 / 24 x 64 products
  const uint32_t m24 = (yb & 0x7FFFFFu) | 0x800000u;
  const uint64_t Y2a = ((uint64_t)m24 * m24) << (14 + 2 * ey);  // y0^2 2^60, exact
  const uint64_t Tma = (3ull << 60) - umulhi_apx(X, Y2a);        // (3 - x y0^2) 2^60
  uint64_t t_hi;
  uint32_t t_lo;
  mul64x32(Tma, m24, t_hi, t_lo);                   // m24 Tm / 2^32
  // y1 2^62 = y0 (3 - x y0^2) / 2 2^62 = m24 Tm 2^(ey - 23 - 60 + 61)
  uint64_t Y = ey >= 0 ? (t_hi << (ey + 10)) | ((uint64_t)t_lo >> (22 - ey))
                       : (t_hi << 9) | ((uint64_t)t_lo >> 23);
  {
    const uint64_t Y2 = umulhi_apx(Y, Y);             // y^2 2^60
    const uint64_t XY2 = umulhi_apx(X, Y2);           // x y^2 2^60
    const uint64_t Tm = (3ull << 60) - XY2;           // (3 - x y^2) 2^60
    Y = umulhi_apx(Y, Tm) << 3;                       // y (3 - x y^2) / 2 2^62
  }
  // sqrt(x) 2^62 (kept below 2^62 + error: no shift, so no wrap near x = 1)
  sq = umulhi_apx(X, Y);
  // sqrt(2L) = sqrt(X 2^E) = sqrt(x) 2^32 2^(E/2) = sq 2^(E/2 - 30)
  se = E / 2 - 30;
}

// |cos|, |sin| of 2 pi x2 2^-53 in 2^-63 fixed point with the signs.
GRNG_BM_HD void sincos_turns(uint64_t x2, uint64_t& c_abs, bool& c_neg, uint64_t& s_abs,
                             bool& s_neg) {
  const uint32_t o = (uint32_t)(x2 >> 50);          // octant
  uint64_t t = x2 & ((1ull << 50) - 1);
  if (o & 1u) t = (1ull << 50) - t;                 // reflect: angle pi/4 - beta
  const uint32_t j = (uint32_t)(t >> 40);           // 0..1024
  const uint64_t h = t & ((1ull << 40) - 1);
  const uint64_t P = umulhi_apx(h << 14, k2Pi61);   // phi 2^64 = 2 pi h 2^11 < 2^53.7
  const uint64_t P2 = umulhi_apx(P, P);             // phi^2 2^64, < 2^43.3
  const uint64_t P3 = umulhi_apx(P2, P);            // < 2^33
  const uint64_t p2s = P2 >> 13;                    // phi^2 2^51, < 2^30.3
  const uint64_t P4 = (p2s * p2s) >> 38;            // phi^4 2^64, < 2^23
  // sin phi = phi - phi^3/6 (+ phi^5/120 < 2^-58) ;
  // 1 - cos phi = phi^2/2 - phi^4/24 (+ phi^6/720 < 2^-71)
  const uint64_t sphi = P - umulhi_apx(P3, kInv6);
  const uint64_t eps = (P2 >> 1) - ((P4 * kInv24_32) >> 32);
  const uint64_t Sj = sint(j), Cj = cost(j);
  const uint64_t sn = Sj - umulhi_apx(Sj, eps) + umulhi_apx(Cj, sphi);  // sin(alpha + phi) 2^63
  const uint64_t cs = Cj - umulhi_apx(Cj, eps) - umulhi_apx(Sj, sphi);  // cos(alpha + phi) 2^63
  const bool swap = ((o + 1u) & 2u) != 0;           // octants 1, 2, 5, 6
  s_abs = swap ? cs : sn;
  c_abs = swap ? sn : cs;
  s_neg = o >= 4u;
  c_neg = ((o + 2u) & 4u) != 0;                     // octants 2, 3, 4, 5
}

// p 2^k as a double, rounded to nearest (ties away), with sign; p = 0 gives +0.
GRNG_BM_HD double assemble(uint64_t p, int k, bool neg) {
  if (p == 0) return 0.0;
  const int nz = clz64(p);
  uint64_t m = p << nz;                             // top bit set
  uint64_t mant = m >> 11;                          // 53 bits
  mant += (m >> 10) & 1u;                           // round half away from zero
  int ex = 63 - nz + k;
  if (mant >> 53) {
    mant >>= 1;
    ex += 1;
  }
  const uint64_t bits = ((uint64_t)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1)) |
                        (neg ? (1ull << 63) : 0ull);
  double d;
  __builtin_memcpy(&d, &bits, 8);
  return d;
}

// The Box-Muller pair for 53-bit x1 (u1 = (x1 + 1) 2^-53) and x2 (u2 = x2 2^-53).
GRNG_BM_HD void box_muller(uint64_t x1, uint64_t x2, double& z0, double& z1) {
  const uint64_t m1 = x1 + 1u;
  uint64_t c_abs, s_abs;
  bool c_neg, s_neg;
  sincos_turns(x2, c_abs, c_neg, s_abs, s_neg);
  if (m1 >> 53) {  // u1 = 1: rho = 0
    z0 = 0.0;
    z1 = 0.0;
    return;
  }
  uint64_t lm, sq;
  int le, se;
  neg_log(m1, lm, le);
  sqrt2x(lm, le, sq, se);
  // z = sq 2^se * c 2^-63 = umulhi(sq, c) 2^(se + 1)
  z0 = assemble(umulhi_apx(sq, c_abs), se + 1, c_neg);
  z1 = assemble(umulhi_apx(sq, s_abs), se + 1, s_neg);
}

}  // namespace bm64
}  // namespace grng
