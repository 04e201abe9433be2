// FP64 Box-Muller in fixed-point integer arithmetic.
//
// The double-precision pipe of this part is narrow (a Box-Muller pair in FP64
// math takes ~60x longer than the same pair's HBM time), so the FP64
// gaussian is computed with 32-bit integer multiplies (plus one FP32 Newton
// step) instead, and only the final result is assembled into an IEEE double
// (round to nearest).
//
//   z0 = rho cos(2 pi u2), z1 = rho sin(2 pi u2), rho = sqrt(-2 ln u1),
//   u1 = (x1 + 1) 2^-53 in (0, 1], u2 = x2 2^-53 in [0, 1), x1, x2 53-bit.
//
// -ln u1:  u1 = 2^-e (1 - delta), delta in (0, 1/2]; a table factor
//          c_i ~ 1/(1 - i/1024) reduces -ln(1 - delta) to ln c_i - ln(1 - r),
//          0 <= r < 2^-9.  The series r + r^2/2 + ... + r^6/6 takes its r^2
//          term from 64-bit products and the r^3..r^6 terms from 32-bit high
//          products of r 2^41 (they need 30 bits or fewer).  When e = 0 and
//          i = 0 (u1 within 2^-10 of 1, -ln u1 below 2^-10) the whole series
//          is evaluated relative to delta instead, so -ln u1 keeps its
//          relative accuracy down to delta = 2^-53.
// rho:     one FP32 Newton step for 1 / sqrt(x) from the hardware estimate,
//          with the residual 1 - x y^2 formed exactly enough by fused
//          multiply-adds (about 2^-43 relative), then sqrt(x) = x y corrected
//          by the residual x - s^2 in fixed point (about 2^-57).
// sincos:  octant symmetry, a 1025-entry table of sin / cos at multiples of
//          2 pi / 8192, the residual angle phi < 2 pi 2^-13 through
//          sin phi = phi - phi^3/6 and 1 - cos phi = phi^2/2 - phi^4/24
//          (the cubic and quartic terms from 32-bit high products), and the
//          rotation by phi as a three-product complex multiply.
// Error budget: below 2^-51 on rho (relative, or absolute when rho < 1) and
// 2^-57 absolute on sin and cos, so |z - exact| stays below about
// 2^-50 max(1, |z|) before the final rounding.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "bm64_tables.h"

#if defined(__CUDACC__)
#define GRNG_BM_HD __host__ __device__ __forceinline__
#else
#define GRNG_BM_HD inline
#endif

namespace grng {
namespace bm64 {

// (sin, cos) and (ln c_i, c_i) are interleaved so that each lookup is one
// 16-byte load.
struct U64Pair {
  uint64_t a, b;
};
#if defined(__CUDACC__)
__device__ const ulonglong2 d_sc[GRNG_BM64_SINT_LEN] = GRNG_BM64_SC;
__device__ const ulonglong2 d_lt[GRNG_BM64_LOGT_LEN] = GRNG_BM64_LT;
__device__ const uint64_t d_e58[GRNG_BM64_E58_LEN] = GRNG_BM64_E58;
__device__ const uint64_t d_exp2t[GRNG_BM64_EXP2T_LEN] = GRNG_BM64_EXP2T;
#endif
static const U64Pair h_sc[GRNG_BM64_SINT_LEN] = GRNG_BM64_SC;
static const U64Pair h_lt[GRNG_BM64_LOGT_LEN] = GRNG_BM64_LT;
static const uint64_t h_e58[GRNG_BM64_E58_LEN] = GRNG_BM64_E58;
static const uint64_t h_exp2t[GRNG_BM64_EXP2T_LEN] = GRNG_BM64_EXP2T;

#if defined(__CUDA_ARCH__)
#define GRNG_BM_TABLE(d, h, i) __ldg(&d[i])
#else
#define GRNG_BM_TABLE(d, h, i) h[i]
#endif
GRNG_BM_HD uint64_t e58(uint32_t e) { return GRNG_BM_TABLE(d_e58, h_e58, e); }
GRNG_BM_HD uint64_t exp2t(uint32_t j) { return GRNG_BM_TABLE(d_exp2t, h_exp2t, j); }
#undef GRNG_BM_TABLE
// sin and cos of 2 pi j / 8192 (2^63 scale)
GRNG_BM_HD void sincos_tab(uint32_t j, uint64_t& s, uint64_t& c) {
#if defined(__CUDA_ARCH__)
  const ulonglong2 v = __ldg(&d_sc[j]);
  s = v.x;
  c = v.y;
#else
  s = h_sc[j].a;
  c = h_sc[j].b;
#endif
}
// ln c_i 2^64 and c_i 2^24
GRNG_BM_HD void log_tab(uint32_t i, uint64_t& t, uint32_t& c) {
#if defined(__CUDA_ARCH__)
  const ulonglong2 v = __ldg(&d_lt[i]);
  t = v.x;
  c = (uint32_t)v.y;
#else
  t = h_lt[i].a;
  c = (uint32_t)h_lt[i].b;
#endif
}

// 32 x 32 -> 64-bit product, and its high word.
GRNG_BM_HD uint64_t mulw(uint32_t a, uint32_t b) { return (uint64_t)a * b; }
GRNG_BM_HD uint32_t mulh(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// High 64 bits of a * b from three 32x32 products: the low x low product and
// the carry out of the low halves of the two cross products are dropped, so
// the result is at most 2 below the exact high word.
GRNG_BM_HD uint64_t umulhi_apx(uint64_t a, uint64_t b) {
  const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
  const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
  return mulw(ah, bh) + mulh(ah, bl) + mulh(al, bh);
}

// High 64 bits of a^2 for a < 2^63: the cross product appears twice, so two
// products suffice (at most 2 below the exact high word).
GRNG_BM_HD uint64_t sqr_hi(uint64_t a) {
  const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
  return mulw(ah, ah) + mulh(ah << 1, al);
}

// Exact 96-bit product of a 64-bit and a 32-bit value: hi = (a c) >> 32,
// lo32 = (a c) mod 2^32.
GRNG_BM_HD void mul64x32(uint64_t a, uint32_t c, uint64_t& hi, uint32_t& lo32) {
  const uint64_t l = mulw((uint32_t)a, c);
  hi = mulw((uint32_t)(a >> 32), c) + (l >> 32);
  lo32 = (uint32_t)l;
}

// Round-to-nearest conversions between uint32 and float.
GRNG_BM_HD float u32_to_f32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __uint2float_rn(x);
#else
  return (float)x;
#endif
}
GRNG_BM_HD uint32_t f32_to_u32_rn(float x) {
#if defined(__CUDA_ARCH__)
  return __float2uint_rn(x);
#else
  return (uint32_t)std::nearbyint(x);
#endif
}

GRNG_BM_HD float bits_f32(uint32_t b) {
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}
GRNG_BM_HD uint32_t f32_bits(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

GRNG_BM_HD int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

GRNG_BM_HD uint32_t clz32(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return (uint32_t)__clz((int)x);
#else
  return (uint32_t)__builtin_clz(x);
#endif
}

// floor(log2 x) for 1 <= x < 2^23: x converts exactly through the 2^23
// shifter, and the float's exponent is the answer (two full-rate
// operations instead of a quarter-rate leading-zero count).
GRNG_BM_HD int ilog2_small(uint32_t x) {
  return (int)(f32_bits(bits_f32(0x4B000000u | x) - 8388608.0f) >> 23) - 127;
}

// High word of (hi:lo) << s and low word of (hi:lo) >> s, for 0 <= s < 32.
GRNG_BM_HD uint32_t shl_hi(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, s);
#else
  return s == 0 ? hi : (hi << s) | (lo >> (32 - s));
#endif
}
GRNG_BM_HD uint32_t shr_lo(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, s);
#else
  return s == 0 ? lo : (lo >> s) | (hi << (32 - s));
#endif
}

GRNG_BM_HD uint64_t join(uint32_t hi, uint32_t lo) { return ((uint64_t)hi << 32) | lo; }

GRNG_BM_HD float fma32(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

GRNG_BM_HD float rsqrt_seed(float x) {
#if defined(__CUDA_ARCH__)
  float y;  // x in [1/4, 1): never subnormal, so the flush-to-zero form
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / std::sqrt(x);
#endif
}

// -ln(u1) for u1 = m1 2^-53, m1 in [1, 2^53), as lm 2^le with lm normalised
// (top bit set).  m1 = 2^53 (u1 = 1) is handled by the caller.
GRNG_BM_HD void neg_log(uint64_t m1, uint64_t& lm, int& le) {
  // M = m1 << s, s = clz(m1): (1 - delta) 2^64 with its top bit set, and
  // u1 = 2^-e (1 - delta) with e = s - 11.  Except when m1 < 2^32
  // (probability 2^-21) the shift is found from the high word alone.
  const uint32_t m1h = (uint32_t)(m1 >> 32), m1l = (uint32_t)m1;
  uint64_t M;
  uint32_t e;
  if (m1h != 0) {
    const uint32_t s = clz32(m1h);          // 11..31 (m1h < 2^21)
    M = join(shl_hi(m1l, m1h, s), m1l << s);
    e = s - 11u;
  } else {
    const int s = clz64(m1);                // 32..63
    M = m1 << s;
    e = (uint32_t)(s - 11);
  }
  const uint64_t D = 0ull - M;              // delta 2^64 in (0, 2^63]
  const uint32_t i = (uint32_t)(D >> 54);   // 0..512
  if (e == 0 && i == 0) {
    // delta < 2^-10: -ln u1 = delta (1 + f), f = delta/2 + delta^2/3 + ... +
    // delta^5/6 (delta^6/7 is below 2^-62 relative), scaled by the
    // normalised delta so that no absolute truncation enters
    const int nz = clz64(D);                // 10..53 (D >= 2^11)
    const uint64_t Dn = D << nz;
    uint64_t G = kInv6;
    G = kInv5 + umulhi_apx(D, G);
    G = kInv4 + umulhi_apx(D, G);
    G = kInv3 + umulhi_apx(D, G);
    G = kInv2 + umulhi_apx(D, G);
    const uint64_t F = umulhi_apx(D, G);    // f 2^64
    const uint64_t half = Dn >> 1;
    const uint64_t Ls = half + umulhi_apx(half, F);  // -ln u1 2^(63 + nz), in [2^62, 2^64)
    const int c = clz64(Ls);                // 0 or 1
    lm = Ls << c;
    le = -63 - nz - c;
    return;
  }
  uint64_t Ti;                              // ln c_i 2^64
  uint32_t C;                               // c_i 2^24
  log_tab(i, Ti, C);
  // r 2^64 = 2^64 - M C 2^-24 (truncating M C 2^-24 leaves r >= 0); the
  // 96-bit product M C is exact, and M C 2^-24 = (hi << 8) | (lo32 >> 24)
  uint64_t mc_hi;
  uint32_t mc_lo;
  mul64x32(M, C, mc_hi, mc_lo);
  const uint64_t R = 0ull - ((mc_hi << 8) | (uint64_t)(mc_lo >> 24));  // < 2^55
  // -ln(1 - r) 2^64 = R + R^2/2 + T3 + T4 + T5 + T6 (r^7/7 < 2^-65.8).
  // With r32 = r 2^41, r^3 comes from 32-bit high products: q = r^2 2^50,
  // t = r^3 2^59.
  const uint32_t r32 = (uint32_t)(R >> 23);
  const uint32_t q = mulh(r32, r32);
  const uint32_t t = mulh(q, r32);
  const uint64_t T3 = mulw(t, 0xAAAAAAABu) >> 28;              // t 2^5 / 3
  // r^4/4 + r^5/5 + r^6/6 stay below 2^26 units of 2^-64, so FP32 is exact
  // enough (error about 4 units) and keeps them off the integer multiplier,
  // the busiest pipe: with x = r 2^9 < 1, 2^64 (r^4/4 + r^5/5 + r^6/6) =
  // x^4 (2^26 + x (2^19/5 + x 2^10/6))
  const float x = u32_to_f32(r32) * 0x1p-32f;
  const float x2 = x * x;
  const uint32_t T456 =
      f32_to_u32_rn(x2 * x2 * fma32(x, fma32(x, 170.66667f, 104857.6f), 67108864.0f));
  const uint64_t S = R + (sqr_hi(R) >> 1) + T3 + T456;
  // -ln(1 - delta) 2^64 = ln c_i 2^64 + S < ln 2 2^64 + 2^55; with e >= 1
  // the sum e ln 2 + ... is kept in units of 2^-58 (below 37 2^58 < 2^64)
  uint64_t Lf = Ti + S;
  int lb = -64;
  if (e != 0) {
    Lf = e58(e) + (Lf >> 6);
    lb = -58;
  }
  // Lf >= 2^54 (-ln u1 >= ln c_1 > 2^-10 here), so its high word is not 0
  const uint32_t Lh = (uint32_t)(Lf >> 32), Ll = (uint32_t)Lf;
  const uint32_t nz = clz32(Lh);            // 0..9 (Lh >= 2^22)
  lm = join(shl_hi(Ll, Lh, nz), Ll << nz);
  le = lb - (int)nz;
}

// sqrt(2 lm 2^le) as sq 2^se, sq in [2^61, 2^62].
GRNG_BM_HD void sqrt2x(uint64_t lm, int le, uint64_t& sq, int& se) {
  int E = le + 1;                           // 2L = lm 2^E
  uint64_t X = lm;
  if (E & 1) {                              // make the exponent even
    X = lm >> 1;
    E += 1;
  }
  // x = X 2^-64 in [1/4, 1) as xh + xl, two 23-bit pieces (error < 2^-46)
  const float xh = bits_f32(0x3F800000u | (uint32_t)(X >> 41)) - 1.0f;
  const float xl = (bits_f32(0x3F800000u | ((uint32_t)(X >> 18) & 0x7FFFFFu)) - 1.0f) * 0x1p-23f;
  // y0 ~ 1/sqrt(x) in [1, 2]; r = 1 - x y0^2 from the exact square
  // y0^2 = p + pe, each fused step rounding at about 2^-46
  const float y0 = rsqrt_seed(xh);
  const float p = y0 * y0;
  const float pe = fma32(y0, y0, -p);
  float r = fma32(-xh, p, 1.0f);
  r = fma32(-xh, pe, r);
  r = fma32(-xl, p, r);
  // y1 = y0 (1 + r/2 + 3 r^2/8): dy = y1 - y0, |dy| < 2^-20, rounded to a
  // multiple of 2^-41 by the 1.5 2^23 shifter
  const float dy = y0 * (r * fma32(0.375f, r, 0.5f));
  const int32_t dyi = (int32_t)(f32_bits(fma32(dy, 0x1p41f, 12582912.0f)) - 0x4B400000u);
  // Y1 = y1 2^62: y0 = m24 2^(ey - 23) with ey = 0 or 1 puts m24 at bit 39 + ey
  const uint32_t yb = f32_bits(y0);
  const uint32_t m24 = (yb & 0x7FFFFFu) | 0x800000u;
  const uint32_t ey = (yb >> 23) - 127u;
  const uint64_t Y1 = join(m24 << (7u + ey), 0u) + (uint64_t)((int64_t)dyi * (int64_t)(1 << 21));
  // s0 = x y1 ~ sqrt(x) 2^62; then s = s0 + (x - s0^2) y1 / 2, in which the
  // residual is at most ~2^-40 x: in 2^-60 units it fits 32 bits, and
  // (x - s0^2) 2^60 y1 / 2 in 2^-62 units is d (y1 2^30) 2^-29
  const uint64_t s0 = umulhi_apx(X, Y1);
  const int32_t d = (int32_t)((uint32_t)(X >> 4) - (uint32_t)sqr_hi(s0));
  const int32_t y30 = (int32_t)(uint32_t)(Y1 >> 32);
  sq = s0 + (uint64_t)(((int64_t)d * (int64_t)y30) >> 29);
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
  const uint64_t P2 = sqr_hi(P);                    // phi^2 2^64 < 2^43.4
  const uint32_t a = (uint32_t)(P2 >> 12);          // phi^2 2^52
  const uint32_t b = (uint32_t)(P >> 22);           // phi 2^42
  // phi^3/6 2^64 = (a b 2^-32) 2/3 needs under 28 significant bits (phi^5/120
  // 2^64 < 41 is dropped)
  // phi^4/24 2^64 = a^2 2^-40 / 24, below 2^18: in FP32 (error below 2^-6)
  const float af = u32_to_f32(a);
  const uint32_t Q4 = f32_to_u32_rn(af * af * 0x1.5555555555556p-45f);
  const uint32_t Q3 = mulh(mulh(a, b), 2863311531u);
  const uint64_t eps = (P2 >> 1) - Q4;              // (1 - cos phi) 2^64
  const uint64_t sphi = P - Q3;                     // sin phi 2^64, >= eps
  // (C + iS)(1 - eps + i sphi) = C + iS + (C + iS)(-eps + i sphi), the last
  // product as k1 = eps (C + S), k2 = C (sphi + eps), k3 = S (sphi - eps):
  // cos = C - k1 - k3, sin = S + k2 - k1
  uint64_t Sj, Cj;
  sincos_tab(j, Sj, Cj);
  const uint64_t k1 = umulhi_apx(Cj + Sj, eps);
  const uint64_t k2 = umulhi_apx(Cj, sphi + eps);
  const uint64_t k3 = umulhi_apx(Sj, sphi - eps);
  const uint64_t cs = Cj - k1 - k3;                 // cos(alpha + phi) 2^63 >= 2^62.5
  const int64_t snv = (int64_t)(Sj + k2 - k1);      // sin(alpha + phi) 2^63, >= -2
  const uint64_t sn = snv < 0 ? 0ull : (uint64_t)snv;
  const bool swap = ((o + 1u) & 2u) != 0;           // octants 1, 2, 5, 6
  s_abs = swap ? cs : sn;
  c_abs = swap ? sn : cs;
  s_neg = o >= 4u;
  c_neg = ((o + 2u) & 4u) != 0;                     // octants 2, 3, 4, 5
}

// p 2^k as a double, rounded to nearest (ties away), with sign; p = 0 gives +0.
// With m = p << s (top bit set), the 53-bit significand is (m >> 11) plus
// the rounding bit (m >> 10) & 1, and the bit pattern is that significand
// plus (E - 1) 2^52, E = 1086 - s + k the biased exponent: the significand's
// leading one supplies the missing 1, and a carry out of rounding (all ones
// rounded up) moves into the exponent by itself.
GRNG_BM_HD double assemble(uint64_t p, int k, bool neg) {
  const uint32_t ph = (uint32_t)(p >> 32), pl = (uint32_t)p;
  uint32_t mh, ml, s;
  if (ph != 0) {
    s = clz32(ph);
    mh = shl_hi(pl, ph, s);
    ml = pl << s;
  } else {                                          // p < 2^32 (|z| < 2^-29)
    if (pl == 0) return 0.0;
    const uint32_t t = clz32(pl);
    s = 32u + t;
    mh = pl << t;
    ml = 0u;
  }
  const uint32_t hi = (mh >> 11) + ((uint32_t)(1085 + k - (int)s) << 20) +
                      (neg ? 0x80000000u : 0u);
  const uint64_t bits = join(hi, shr_lo(ml, mh, 11)) + ((ml >> 10) & 1u);
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}

// The Box-Muller pair in fixed point: z0 = (n0 ? -p0 : p0) 2^k,
// z1 = (n1 ? -p1 : p1) 2^k, p0, p1 < 2^62; u1 = 1 gives p0 = p1 = 0.
struct FixedPair {
  uint64_t p0, p1;
  int k;
  bool n0, n1;
};

// The Box-Muller pair for 53-bit x1 (u1 = (x1 + 1) 2^-53) and x2 (u2 = x2 2^-53).
GRNG_BM_HD FixedPair box_muller_fixed(uint64_t x1, uint64_t x2) {
  const uint64_t m1 = x1 + 1u;
  uint64_t c_abs, s_abs;
  bool c_neg, s_neg;
  sincos_turns(x2, c_abs, c_neg, s_abs, s_neg);
  FixedPair r;
  r.n0 = c_neg;
  r.n1 = s_neg;
  if (m1 >> 53) {  // u1 = 1: rho = 0
    r.p0 = r.p1 = 0;
    r.k = 0;
    return r;
  }
  uint64_t lm, sq;
  int le, se;
  neg_log(m1, lm, le);
  sqrt2x(lm, le, sq, se);
  // z = sq 2^se * c 2^-63 = umulhi(sq, c) 2^(se + 1)
  r.p0 = umulhi_apx(sq, c_abs);
  r.p1 = umulhi_apx(sq, s_abs);
  r.k = se + 1;
  return r;
}

GRNG_BM_HD void box_muller(uint64_t x1, uint64_t x2, double& z0, double& z1) {
  const FixedPair f = box_muller_fixed(x1, x2);
  z0 = assemble(f.p0, f.k, f.n0);
  z1 = assemble(f.p1, f.k, f.n1);
}

// exp(m + s z) for z = (neg ? -p : p) 2^k, written exp(m) 2^(s z log2 e):
// exp(m) = em_mant 2^em_exp (em_mant normalised) and s = s_mant 2^s_exp
// (s_mant the 53-bit significand) are prepared per launch on the host.
// V = s z log2 e splits into n + f, f in [0, 1); 2^f = 2^(j/256) e^t with a
// 257-entry table and t = (f - j/256) ln 2 < 2^-8.5, e^t - 1 summed to t^5
// (t^6/720 < 2^-60; t^3..t^5 from 32-bit high products of t 2^40).  Returns
// false, leaving the output to the caller's FP64 path, when |V| >= 2^11 or
// the result is not a normal double.  Error: below 2^-51 relative besides
// the error of z itself, which s z log2 e carries into the exponent.
GRNG_BM_HD bool lognormal_fixed(uint64_t p, int k, bool neg, uint64_t em_mant, int em_exp,
                                uint64_t s_mant, int s_exp, double& out) {
  const uint64_t W = umulhi_apx(s_mant << 11, p);          // |s z| = W 2^(k + s_exp + 53)
  const uint64_t W2 = umulhi_apx(W, kLog2e63);             // |V| = W2 2^(k + s_exp + 54)
  const int sh = k + s_exp + 54 + 52;                      // A = |V| 2^52 = W2 2^sh
  uint64_t A;
  if (sh >= 0) {
    if (sh >= 63 || (W2 >> (63 - sh)) != 0) return false;   // |V| >= 2^11
    A = W2 << sh;
  } else {
    A = sh <= -64 ? 0ull : (W2 >> (-sh));
  }
  // V = n + f with f = F 2^-52 in [0, 1)
  const int nabs = (int)(A >> 52);
  uint64_t F = A & ((1ull << 52) - 1);
  int n = nabs;
  if (neg && A != 0) {
    if (F != 0) {
      n = -nabs - 1;
      F = (1ull << 52) - F;
    } else {
      n = -nabs;
    }
  }
  const uint32_t j = (uint32_t)(F >> 44);
  const uint64_t G = F & ((1ull << 44) - 1);               // (f - j/256) 2^52
  const uint64_t T = umulhi_apx(G << 20, kLn2) >> 8;       // t 2^64 < 2^55.5
  const uint32_t t40 = (uint32_t)(T >> 24);                // t 2^40
  const uint32_t q = mulh(t40, t40);                       // t^2 2^48
  const uint32_t c = mulh(q, t40);                         // t^3 2^56
  const uint32_t d = mulh(q, q);                           // t^4 2^64
  const uint32_t e5 = mulh(d, t40);                        // t^5 2^72
  const uint64_t Ex = T + (sqr_hi(T) >> 1) + (mulw(c, 0x2AAAAAABu) >> 24) +  // t + t^2/2 + t^3/6
                      mulh(d, 0x0AAAAAABu) + (mulh(e5, 0x02222222u) >> 8);  // + t^4/24 + t^5/120
  const uint64_t P = exp2t(j);                             // 2^(j/256) 2^62
  const uint64_t M = P + umulhi_apx(P, Ex);                // 2^f 2^62 in [2^62, 2^63]
  const uint64_t R = umulhi_apx(em_mant, M);               // exp(m) 2^f = R 2^(em_exp + 2)
  const int kk = em_exp + 2 + n;                           // R in [2^61, 2^63)
  if (kk + 62 > 1023 || kk + 61 < -1022) return false;
  out = assemble(R, kk, false);
  return true;
}

#if !defined(__CUDA_ARCH__)
// Host side of lognormal_fixed: exp(m) and s split for a launch; false when
// the fixed-point path is not used: |m| > 11000 (every output is then 0 or
// infinite) or s outside [2^-60, 2^20].  exp(m) keeps an integer exponent,
// so m + s z may lie anywhere in the double range.
inline bool lognormal_consts(double m, double s, uint64_t& em_mant, int& em_exp,
                             uint64_t& s_mant, int& s_exp) {
  if (!(std::fabs(m) <= 11000.0) || !(s >= 0x1p-60) || !(s <= 0x1p20)) return false;
  int ex = 0;
  const long double fr = std::frexp(std::exp((long double)m), &ex);  // [1/2, 1)
  const long double scaled = std::ldexp(fr, 64);                      // [2^63, 2^64)
  long double hi = std::floor(scaled);
  uint64_t mant = (uint64_t)hi;
  if (scaled - hi >= 0.5L) {
    if (mant == ~0ull) {
      mant = 1ull << 63;
      ex += 1;
    } else {
      mant += 1;
    }
  }
  em_mant = mant;
  em_exp = ex - 64;
  int es = 0;
  const double fs = std::frexp(s, &es);                               // [1/2, 1)
  s_mant = (uint64_t)std::ldexp(fs, 53);
  s_exp = es - 53;
  return true;
}
#endif

}  // namespace bm64
}  // namespace grng
