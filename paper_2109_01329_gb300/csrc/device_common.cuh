// Device-side building blocks shared by the Philox and MRG32k3a fill kernels:
// the Philox4x32-10 bijection, exact word -> uniform conversions, the fused
// range transform and the Box-Muller / lognormal transforms.
#pragma once

#include <cstdint>

#include "bm64_fixed.cuh"
#include "grng_internal.h"
#include "icdf32_tables.h"
#include "icdf64_fixed.cuh"

namespace grng {
namespace dev {

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Per round: the two
// 32x32 -> 64-bit products of counter words 0 and 2 with fixed multipliers;
// the high halves are mixed with counter words 1, 3 and the round key, the
// low halves move to words 1 and 3.  The key advances by two Weyl constants
// between rounds.  The round keys are warp-uniform, so the compiler keeps
// them in uniform registers.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
    const uint32_t lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// The ten round keys of one key, (k0 + r W0, k1 + r W1) for r = 0..9, made
// once per launch on the host.  Kept in a kernel's parameter space, each
// round's key is a constant-bank operand of its XOR, so the key schedule
// costs no instruction in the loop.
struct PhiloxRoundKeys {
  uint32_t k[20];
};
__host__ __device__ inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxRoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0 + (uint32_t)r * kPhiloxW0;
    rk.k[2 * r + 1] = k1 + (uint32_t)r * kPhiloxW1;
  }
  return rk;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
    const uint32_t lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk.k[2 * r], lo1, hi0 ^ c.w ^ rk.k[2 * r + 1], lo0);
  }
  return c;
}

// Philox counter of a block index given as (lo, hi) 64-bit halves.  Word
// offsets live in Z / 2^128, so block indices live in Z / 2^126: the top two
// bits are cleared, which makes word 2^128 + g equal to word g.
__device__ __forceinline__ uint4 ctr_from(uint64_t lo, uint64_t hi) {
  return make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi,
                    (uint32_t)(hi >> 32) & 0x3FFFFFFFu);
}

// (lo, hi) += v with carry.
__device__ __forceinline__ void add128(uint64_t& lo, uint64_t& hi, uint64_t v) {
  const uint64_t s = lo + v;
  hi += (s < lo) ? 1u : 0u;
  lo = s;
}

// ------------------------------------------------------------ conversions
// u = (w >> 8) 2^-24: the 24-bit integer converts exactly, the scale is exact.
__device__ __forceinline__ float u01_f32(uint32_t w) {
  return __uint2float_rn(w >> 8) * 0x1p-24f;
}

// x 2^e for an integer 0 <= x <= 2^53, built with integer operations only
// (exact: x has at most 53 significant bits, or is 2^53, and the result is a
// normal double for the exponents used here).  Avoids the FP64 pipe, which
// is narrow on this part.
__device__ __forceinline__ double scaled_u54_to_f64(uint64_t x, int e) {
  if (x == 0) return 0.0;
  const int lz = __clzll((long long)x);
  const int msb = 63 - lz;
  const uint64_t frac = ((x << lz) << 1) >> 12;  // drop the leading one, keep 52 bits
  const uint64_t bexp = (uint64_t)(1023 + msb + e);
  return __longlong_as_double((long long)((bexp << 52) | frac));
}

// Signed form: v 2^e for |v| <= 2^53.  The sign goes in as a bit: negating
// the double would be an FP64 instruction.
__device__ __forceinline__ double scaled_i54_to_f64(int64_t v, int e) {
  const uint64_t mag = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
  const uint64_t bits = (uint64_t)__double_as_longlong(scaled_u54_to_f64(mag, e));
  return __longlong_as_double((long long)(bits | (v < 0 ? (1ull << 63) : 0ull)));
}

// The 53-bit integer of an FP64 uniform: ((w_a << 32) | w_b) >> 11.
__device__ __forceinline__ uint64_t u53(uint32_t wa, uint32_t wb) {
  return ((((uint64_t)wa) << 32) | (uint64_t)wb) >> 11;
}

// The FP64 uniform x 2^-53, x = u53(w_a, w_b), in 32-bit halves.  Unless
// x < 2^32 (probability 2^-21) the leading one of x lies in its top 21 bits
// h = w_a >> 11: with c = clz(h) and s = c - 11, m = x << s has it at bit 52
// and x 2^-53 = m 2^(-53 - s), whose bit pattern is m + (1021 - s) 2^52 =
// m + (1032 - c) 2^52 (the leading one of m adds the missing 1 to the biased
// exponent 1022 - s).  The leading-zero count runs on the special-function
// pipe, which the uniform fills leave idle, in place of four integer and
// FP32 operations.  Same value as scaled_u54_to_f64(x, -53).
__device__ __forceinline__ double u01_f64(uint32_t wa, uint32_t wb) {
  const uint32_t h = wa >> 11;
  const uint32_t l = __funnelshift_r(wb, wa, 11);  // low 32 bits of x
  if (h == 0) return scaled_u54_to_f64((uint64_t)l, -53);
  const uint32_t c = (uint32_t)__clz((int)h);      // 11..31
  const uint32_t s = c - 11u;                      // 0..20
  const uint32_t mh = __funnelshift_l(l, h, s);    // high half of x << s
  const uint32_t ml = l << s;
  return __hiloint2double((int)(mh + (1032u << 20) - (c << 20)), (int)ml);
}

// d u rounded to nearest (even), u = x 2^-53, x = (xh 2^32 + xl) with
// xh != 0, for d = D 2^e (D = rd_hi 2^32 + rd_lo in [2^52, 2^53)), whose
// nonzero products are normal doubles (checked on the host): the same value
// as the FP64 multiply, from four 32 x 32 products.  With X = x << s in
// [2^52, 2^53), P = D X lies in [2^104, 2^106); its top 53 bits, rounded on
// the next bit and the OR of all lower ones (ties to even), are the
// significand m, and the bit pattern is m + (E - 1) 2^52 (the leading one of
// m completes the biased exponent E; a carry out of rounding moves into the
// exponent by itself).
__device__ __forceinline__ double mul_rn_u53(uint32_t xh, uint32_t xl, const TransformParams& t) {
  const uint32_t c = (uint32_t)__clz((int)xh);      // 11..31
  const uint32_t s = c - 11u;
  const uint32_t Xh = __funnelshift_l(xl, xh, s);   // [2^20, 2^21)
  const uint32_t Xl = xl << s;
  const uint64_t LL = (uint64_t)t.rd_lo * Xl;
  const uint64_t M = (uint64_t)t.rd_lo * Xh + (uint64_t)t.rd_hi * Xl;  // < 2^54
  const uint64_t mid = (LL >> 32) + (M & 0xFFFFFFFFull);                // < 2^33
  const uint32_t w0 = (uint32_t)LL;
  const uint32_t w1 = (uint32_t)mid;
  const uint64_t U = (uint64_t)t.rd_hi * Xh + (M >> 32) + (mid >> 32);  // P >> 64
  const bool top = (U >> 41) != 0;                                      // P >= 2^105
  const uint32_t q = top ? 11u : 12u;
  const uint64_t m0 = (U << q) | (uint64_t)(w1 >> (32u - q));           // P >> (64 - q)
  const uint32_t rb = (w1 >> (31u - q)) & 1u;
  const uint32_t sticky = (w1 & ((1u << (31u - q)) - 1u)) | w0;
  const uint64_t m = m0 + (uint64_t)(rb & ((sticky != 0u) | (uint32_t)(m0 & 1u)));
  // t = m 2^(e - s) (top) or m 2^(e - s - 1): E = that exponent + 1075
  const int64_t E = (int64_t)t.rd_exp - (int64_t)s - (top ? 0 : 1) + 1075;
  return __longlong_as_double((long long)(m + ((uint64_t)(E - 1) << 52)));
}

// The same value with one FP64 add in place of the normalisation: with B the
// double whose bits are 0x3FE 2^52 + (x mod 2^52), i.e. 1/2 + (x mod 2^52)
// 2^-53, x 2^-53 is B when x >= 2^52 and B - 1/2 otherwise, both exact (no
// rare path).  The fills use it for every second unit, so the otherwise idle
// FP64 pipe takes half the conversions off the integer pipes.
__device__ __forceinline__ double u01_f64_dadd(uint32_t wa, uint32_t wb) {
  const uint32_t h = wa >> 11;                      // x >> 32: 21 bits
  const uint32_t l = __funnelshift_r(wb, wa, 11);   // low 32 bits of x
  const double B = __hiloint2double((int)((h & 0xFFFFFu) | 0x3FE00000u), (int)l);
  return __dadd_rn(B, (h >> 20) != 0u ? 0.0 : -0.5);
}

// ---------------------------------------------------------- range transform
// Sec. 4.3, Listing 2 computes acc * (b - a) + a in a second kernel; here it
// is fused, with explicit round-to-nearest multiply and add (never
// contracted into an FMA) and the half-open interval enforced.
__device__ __forceinline__ float range_f32(float u, const TransformParams& t) {
  const float r = __fadd_rn(t.fa, __fmul_rn(t.fd, u));
  return r >= t.fb ? t.fbprev : r;
}
// The FP64 form for the words (w_a, w_b) of x: the product in integers (one
// FP64 operation, the add, remains; a product, add and compare on this
// part's narrow FP64 pipe took 3.4x the [0, 1) fill's time), the clamp as
// the host's threshold on x.  x < 2^32 (probability 2^-21) and ranges whose
// products can leave the normal doubles take the FP64 product.
// kInt = false takes the FP64 product for every x: the fill kernels pass it
// for every second unit, so the integer pipes and the FP64 pipe share the
// products (a constant after unrolling; both forms give the same bits).
template <bool kInt>
__device__ __forceinline__ double uniform_ab_f64(uint32_t wa, uint32_t wb,
                                                 const TransformParams& t) {
  const uint32_t xh = wa >> 11;
  const uint32_t xl = __funnelshift_r(wb, wa, 11);
  double prod;
  if (kInt && t.r_int != 0 && xh != 0) {
    prod = mul_rn_u53(xh, xl, t);
  } else {
    prod = __dmul_rn(t.dd, u01_f64(wa, wb));
  }
  const double r = __dadd_rn(t.da, prod);
  const uint64_t x = ((uint64_t)xh << 32) | xl;
  return x >= t.r_xthr ? t.dbprev : r;
}

// -------------------------------------------------------------- Box-Muller
// FP32 pieces from the exact integers of u1 and u2; the polynomial
// coefficients come from gen_bm32_poly.py (fits on Chebyshev nodes refined
// towards minimax, rounded to float).
//
// -2 ln(j 2^-24) for j in [1, 2^24] (the Box-Muller u1 has j = (w >> 8) + 1): j = 2^e m with m
// in [sqrt(1/2), sqrt(2)) split from the float's bits, t = m - 1 (exact),
// ln m = t + t^2 P(t) (P of degree 7, relative error below 3e-8), and
// -2 ln u1 = 2 ((24 - e) ln 2 - ln m): no cancellation as u1 -> 1 (e = 24).
// Over all 2^24 inputs the relative error stays below 1e-7.
__device__ __forceinline__ float neg2_log_j_f32(uint32_t j) {
  const float f = __uint2float_rn(j);  // exact
  const int ix = __float_as_int(f);
  const int e = (ix - 0x3F3504F3) >> 23;
  const float t = __int_as_float(ix - (e << 23)) - 1.0f;
  float p = 0.08734750747680664f;
  p = fmaf(p, t, -0.14307482540607452f);
  p = fmaf(p, t, 0.14917989075183868f);
  p = fmaf(p, t, -0.165705144405365f);
  p = fmaf(p, t, 0.19962070882320404f);
  p = fmaf(p, t, -0.25001755356788635f);
  p = fmaf(p, t, 0.33333951234817505f);
  p = fmaf(p, t, -0.49999991059303284f);
  const float lnm = fmaf(t * t, p, t);
  // 24 - e in [0, 24] as a float by the 2^23 shifter
  const float k = __int_as_float(0x4B000000 + 24 - e) - 8388608.0f;
  return 2.0f * fmaf(k, 0.693147182464599609375f, -lnm);
}
__device__ __forceinline__ float neg2_log_u1_f32(uint32_t w) { return neg2_log_j_f32((w >> 8) + 1u); }

// sin and cos of 2 pi k 2^-24, k = w >> 8: octant o = k >> 21, the position
// t in [0, 2^21] within it (reflected in odd octants), v = t 2^-21 (exact),
// sin(pi v / 4) = v S(v^2) and cos(pi v / 4) = 1 + v^2 C(v^2) (fit errors
// 2.4e-9 relative and 5.4e-11); at most 8.5e-8 from the exact values over
// all 2^24 angles.
__device__ __forceinline__ void sincos_turns_f32(uint32_t w, float& s, float& c) {
  const uint32_t k = w >> 8;
  const uint32_t o = k >> 21;
  uint32_t t = k & 0x1FFFFFu;
  if (o & 1u) t = 0x200000u - t;
  const float v = (__int_as_float(0x4B000000u | t) - 8388608.0f) * 0x1p-21f;
  const float ww = v * v;
  const float sn =
      v * fmaf(fmaf(fmaf(-3.595459565985948e-05f, ww, 0.0024900073185563087f), ww,
                    -0.08074543625116348f),
               ww, 0.7853981852531433f);
  const float cs =
      fmaf(ww,
           fmaf(fmaf(fmaf(3.531334868966951e-06f, ww, -0.00032594200456514955f), ww,
                     0.015854327008128166f),
                ww, -0.3084251284599304f),
           1.0f);
  const bool swap = ((o + 1u) & 2u) != 0;  // octants 1, 2, 5, 6
  const float a = swap ? cs : sn, b = swap ? sn : cs;
  s = (o >= 4u) ? -a : a;
  c = (((o + 2u) & 4u) != 0) ? -b : b;  // octants 2, 3, 4, 5
}

// FP32 inverse CDF of the standard normal for u = (k + 1/2) 2^-23, k = w >> 9
// (polynomials in icdf32_tables.h, written by gen_icdf32_tables.py).  With
// x = 2u - 1 = (2k + 1 - 2^23) 2^-23 (exact) and v = -log2(1 - x^2),
// Phi^-1(u) = sqrt(2) erfinv(x) = x P(v): P1(v) of degree 9 below
// v = 5 / ln 2 (|x| < 0.9966, 99.7% of outputs, so warps rarely diverge) and
// P2(sqrt(v) - sqrt(5 / ln 2)) of degree 8 above (Giles's form of erfinv).
// 1 - x^2 comes from one FMA of the exact x (one rounding) and v from the
// hardware lg2.approx (flush-to-zero form: q is never subnormal).  z depends
// on v only through x P'(v), so the absolute error of lg2.approx (about
// 2^-22) moves z by a few 1e-8: emulated over all 2^23 inputs with twice that
// log error the result stays within 2.2e-7 of max(1, |z|) from the exact
// value.  The central polynomial runs for every input, so that a thread's
// several inverse CDFs are straight-line code; the rare tail input redoes r
// afterwards.
struct Icdf32 {
  float x, v, r;
};
__device__ __forceinline__ Icdf32 icdf_f32_central(uint32_t w) {
  Icdf32 c;
  // 2^23 + k by the 2^23 shifter, then x = (k 2^-22 - 1) + 2^-23: both steps exact
  const float f = __int_as_float(0x4B000000u | (w >> 9));
  c.x = fmaf(f, 0x1p-22f, -3.0f) + 0x1p-23f;
  const float q = fmaf(-c.x, c.x, 1.0f);  // 1 - x^2 in [2^-22, 1]
  float lg;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(q));
  c.v = -lg;
  c.r = GRNG_ICDF32_P1(c.v);
  return c;
}
__device__ __forceinline__ bool icdf_f32_is_tail(const Icdf32& c) { return c.v >= GRNG_ICDF32_V1; }
__device__ __forceinline__ void icdf_f32_tail(Icdf32& c) {
  float sv;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sv) : "f"(c.v));
  const float d = sv - GRNG_ICDF32_SQRT_V1;
  c.r = GRNG_ICDF32_P2(d);
}
__device__ __forceinline__ float icdf_f32_finish(const Icdf32& c) { return c.x * c.r; }
__device__ __forceinline__ float icdf_f32(uint32_t w) {
  Icdf32 c = icdf_f32_central(w);
  if (icdf_f32_is_tail(c)) icdf_f32_tail(c);
  return icdf_f32_finish(c);
}

// rho = sqrt(-2 ln u1) by the hardware square root (relative error about
// 2^-23; its argument is 0 or at least -2 ln(1 - 2^-24) > 1e-7, never
// subnormal, so the flush-to-zero form, which skips the subnormal handling),
// z0 = rho cos(2 pi u2), z1 = rho sin(2 pi u2).
__device__ __forceinline__ void box_muller_f32(uint32_t w0, uint32_t w1, float& z0, float& z1) {
  const float v = neg2_log_u1_f32(w0);
  float rho;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rho) : "f"(v));
  float s, c;
  sincos_turns_f32(w1, s, c);
  z0 = rho * c;
  z1 = rho * s;
}

// FP64 pair: integer fixed-point evaluation (see bm64_fixed.cuh), within
// about 1 ulp of the exact value, without the FP64 pipe.
__device__ __forceinline__ void box_muller_f64(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                               double& z0, double& z1) {
  bm64::box_muller(u53(w0, w1), u53(w2, w3), z0, z1);
}

// mean + sd z, or exp of it, as the output word of an inverse-CDF variant
template <int V>
__device__ __forceinline__ uint32_t icdf_out_f32(float z, const TransformParams& t) {
  float y = fmaf(t.fsd, z, t.fmean);
  if constexpr (V == V_ICDF_LOGN_F32) y = expf(y);
  return __float_as_uint(y);
}

// ------------------------------------------------- one unit -> its outputs
// Writes the output words (4 bytes each) of one unit from its words.
// odd: the unit's index in its block or chunk is odd (only the F64 uniforms
// look at it, to alternate the integer and the FP64 pipe)
template <int V>
__device__ __forceinline__ void unit_outputs(const uint32_t* w, uint32_t* o,
                                             const TransformParams& t, bool odd = false) {
  if constexpr (V == V_BITS) {
    o[0] = w[0];
  } else if constexpr (V == V_U01_F32) {
    o[0] = __float_as_uint(u01_f32(w[0]));
  } else if constexpr (V == V_UNI_F32) {
    o[0] = __float_as_uint(range_f32(u01_f32(w[0]), t));
  } else if constexpr (V == V_U01_F64 || V == V_AFF_F64 || V == V_UNI_F64) {
    double r;
    if constexpr (V == V_U01_F64) {
      r = odd ? u01_f64_dadd(w[0], w[1]) : u01_f64(w[0], w[1]);
    } else if constexpr (V == V_AFF_F64) {
      r = scaled_i54_to_f64(t.aff_a + (int64_t)u53(w[0], w[1]), t.aff_exp);
    } else {
      r = odd ? uniform_ab_f64<false>(w[0], w[1], t) : uniform_ab_f64<true>(w[0], w[1], t);
    }
    const uint64_t b = (uint64_t)__double_as_longlong(r);
    o[0] = (uint32_t)b;
    o[1] = (uint32_t)(b >> 32);
  } else if constexpr (V == V_GAUSS_F32 || V == V_LOGN_F32) {
    float z0, z1;
    box_muller_f32(w[0], w[1], z0, z1);
    float y0 = fmaf(t.fsd, z0, t.fmean);
    float y1 = fmaf(t.fsd, z1, t.fmean);
    if constexpr (V == V_LOGN_F32) {
      y0 = expf(y0);
      y1 = expf(y1);
    }
    o[0] = __float_as_uint(y0);
    o[1] = __float_as_uint(y1);
  } else if constexpr (V == V_ICDF_GAUSS_F32 || V == V_ICDF_LOGN_F32) {
    // u = (k + 1/2) 2^-23, k = w >> 9: an exact midpoint in (0, 1)
    o[0] = icdf_out_f32<V>(icdf_f32(w[0]), t);
  } else if constexpr (V == V_ICDF_GAUSS_F64 || V == V_ICDF_LOGN_F64) {
    // u = (x + 1/2) 2^-52, x = ((w_a << 32) | w_b) >> 12; Phi^-1 in fixed
    // point (icdf64_fixed.cuh), then mean + sd z or exp(m + s z) as for the
    // Box-Muller outputs
    const uint64_t x = ((((uint64_t)w[0]) << 32) | (uint64_t)w[1]) >> 12;
    bool neg;
    const uint64_t t59 = icdf64::icdf_t59(x, neg);
    double y;
    if constexpr (V == V_ICDF_GAUSS_F64) {
      y = fma(t.dsd, bm64::assemble(t59, -59, neg), t.dmean);
    } else {
      if (!(t.ln_fast && bm64::lognormal_fixed(t59, -59, neg, t.ln_em_mant, t.ln_em_exp,
                                               t.ln_s_mant, t.ln_s_exp, y)))
        y = exp(fma(t.dsd, bm64::assemble(t59, -59, neg), t.dmean));
    }
    const uint64_t b = (uint64_t)__double_as_longlong(y);
    o[0] = (uint32_t)b;
    o[1] = (uint32_t)(b >> 32);
  } else if constexpr (V == V_LOGN_F64) {
    // exp(m + s z) in fixed point from the fixed-point pair (no FP64
    // instruction); an output outside its range takes the FP64 path
    const bm64::FixedPair f = bm64::box_muller_fixed(u53(w[0], w[1]), u53(w[2], w[3]));
    double y0, y1;
    if (!(t.ln_fast && bm64::lognormal_fixed(f.p0, f.k, f.n0, t.ln_em_mant, t.ln_em_exp,
                                             t.ln_s_mant, t.ln_s_exp, y0)))
      y0 = exp(fma(t.dsd, bm64::assemble(f.p0, f.k, f.n0), t.dmean));
    if (!(t.ln_fast && bm64::lognormal_fixed(f.p1, f.k, f.n1, t.ln_em_mant, t.ln_em_exp,
                                             t.ln_s_mant, t.ln_s_exp, y1)))
      y1 = exp(fma(t.dsd, bm64::assemble(f.p1, f.k, f.n1), t.dmean));
    const uint64_t b0 = (uint64_t)__double_as_longlong(y0);
    const uint64_t b1 = (uint64_t)__double_as_longlong(y1);
    o[0] = (uint32_t)b0;
    o[1] = (uint32_t)(b0 >> 32);
    o[2] = (uint32_t)b1;
    o[3] = (uint32_t)(b1 >> 32);
  } else {  // V_GAUSS_F64, V_STDGAUSS_F64
    double z0, z1;
    box_muller_f64(w[0], w[1], w[2], w[3], z0, z1);
    double y0 = z0, y1 = z1;
    // (0, 1) is its own variant rather than a run-time branch: a branch over
    // the two FP64 multiply-adds is predicated, and they would still issue
    // on the narrow FP64 pipe
    if constexpr (V != V_STDGAUSS_F64) {
      y0 = fma(t.dsd, z0, t.dmean);
      y1 = fma(t.dsd, z1, t.dmean);
    }
    const uint64_t b0 = (uint64_t)__double_as_longlong(y0);
    const uint64_t b1 = (uint64_t)__double_as_longlong(y1);
    o[0] = (uint32_t)b0;
    o[1] = (uint32_t)(b0 >> 32);
    o[2] = (uint32_t)b1;
    o[3] = (uint32_t)(b1 >> 32);
  }
}

// Output words of one 4-word block whose 4 words are exactly the words of
// 4 / wpu whole units (the aligned case).
template <int V>
__device__ __forceinline__ uint4 block_outputs(uint4 b, const TransformParams& t) {
  constexpr int kWpu = (V == V_BITS || V == V_U01_F32 || V == V_UNI_F32 ||
                        V == V_ICDF_GAUSS_F32 || V == V_ICDF_LOGN_F32)
                           ? 1
                       : (V == V_GAUSS_F64 || V == V_LOGN_F64 || V == V_STDGAUSS_F64) ? 4
                                                                 : 2;
  uint32_t w[4] = {b.x, b.y, b.z, b.w};
  uint32_t o[4];
  if constexpr (V == V_ICDF_GAUSS_F32 || V == V_ICDF_LOGN_F32) {
    // the four central evaluations interleave; one vote skips the tails
    Icdf32 c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = icdf_f32_central(w[u]);
    if (icdf_f32_is_tail(c[0]) | icdf_f32_is_tail(c[1]) | icdf_f32_is_tail(c[2]) |
        icdf_f32_is_tail(c[3])) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (icdf_f32_is_tail(c[u])) icdf_f32_tail(c[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = icdf_out_f32<V>(icdf_f32_finish(c[u]), t);
  } else {
#pragma unroll
    for (int u = 0; u < 4 / kWpu; ++u) unit_outputs<V>(w + u * kWpu, o + u * kWpu, t, (u & 1) != 0);
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

template <int V>
struct VInfo {
  static constexpr int wpu = (V == V_BITS || V == V_U01_F32 || V == V_UNI_F32 ||
                              V == V_ICDF_GAUSS_F32 || V == V_ICDF_LOGN_F32)
                                 ? 1
                             : (V == V_GAUSS_F64 || V == V_LOGN_F64 || V == V_STDGAUSS_F64) ? 4
                                                                       : 2;
  static constexpr int es = (V == V_BITS || V == V_U01_F32 || V == V_UNI_F32 ||
                             V == V_GAUSS_F32 || V == V_LOGN_F32 || V == V_ICDF_GAUSS_F32 ||
                             V == V_ICDF_LOGN_F32)
                                ? 4
                                : 8;
  static constexpr int epu = (V == V_GAUSS_F32 || V == V_LOGN_F32 || V == V_GAUSS_F64 ||
                              V == V_LOGN_F64 || V == V_STDGAUSS_F64)
                                 ? 2
                                 : 1;
  static constexpr int ow_per_elem = es / 4;  // output words per element
  // instruction weight of one unit: 0 a few operations, 1 a single-precision
  // log / sincos / inverse CDF, 2 the fixed-point FP64 Box-Muller, inverse
  // CDF or lognormal (hundreds of instructions); loops
  // over units unroll less as the weight grows, so a loop body stays in the
  // instruction cache
  static constexpr int weight =
      (V == V_GAUSS_F64 || V == V_LOGN_F64 || V == V_STDGAUSS_F64 || V == V_ICDF_GAUSS_F64 ||
       V == V_ICDF_LOGN_F64)
          ? 2
      : (V == V_GAUSS_F32 || V == V_LOGN_F32 || V == V_ICDF_GAUSS_F32 || V == V_ICDF_LOGN_F32)
          ? 1
          : 0;
};

// 16-byte vector store (the address must be 16-byte aligned).
__device__ __forceinline__ void store16(void* p, uint4 v) {
  *reinterpret_cast<uint4*>(p) = v;
}

}  // namespace dev
}  // namespace grng
