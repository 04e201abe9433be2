// grng oracle: a plain, slow, sequential CPU reference of the random number
// generation path (engine -> words -> distribution transform).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
// loads this file.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline leg use it.  It shares no code, header, table or constant
// generator with the CUDA path: every constant below is restated here from
// the published definitions.
//
// What the paper fixes and what it leaves open:
//   * Sec. 4.1 names the two engine families (Philox4x32x10 and an MRG) and
//     the oneMKL engine / distribution / generate(distr, engine, n, r)
//     interface; Sec. 4.2 names seed and offset as generator options.
//   * Sec. 4.3, Listing 2 gives the range transform r * (b - a) + a.
//   * Everything else (the generator definitions, seeding, word -> float
//     conversion, Box-Muller pairing) is not in the paper.  The readings taken
//     here are:
//       - Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw (SC'11):
//         key (k0, k1) = (seed mod 2^32, seed >> 32); the 128-bit counter of
//         word g is floor(g / 4), word g is lane g mod 4 of that block.
//       - MRG32k3a as published by L'Ecuyer (1999): the seeded state is
//         x1 = (1, 1, seed mod m1), x2 = (1, 1, 1) as (x_{-3}, x_{-2}, x_{-1});
//         word n is z_n = (x1_n - x2_n) mod m1 after step n (n = 0, 1, ...).
//       - uniform FP32: u = (w >> 8) * 2^-24; FP64: u = ((w_a<<32|w_b)>>11) * 2^-53
//         with w_a the earlier word.
//       - [a, b): r = a + (b - a) * u, each operation rounded to nearest in the
//         output type (no fused multiply-add); r >= b becomes the largest
//         value below b.  Parameters are first rounded to the output type.
//       - Box-Muller: consecutive pairs; u1 is the (0,1] variant of the first
//         uniform, u2 the [0,1) uniform of the second; z0 = rho cos(2 pi u2),
//         z1 = rho sin(2 pi u2), rho = sqrt(-2 ln u1); gaussian = mean + sd z,
//         lognormal = exp(m + s z).  An odd n still consumes the last pair.
//       - ICDF method (oneMKL's icdf gaussian / lognormal, Sec. 4.1): one
//         open-interval uniform per output, u = (k + 1/2) 2^-23, k = w >> 9
//         (FP32) or u = (x + 1/2) 2^-52, x = ((w_a << 32 | w_b) >> 12) (FP64);
//         z = Phi^-1(u), found by bisection and Newton steps on
//         Phi(z) = erfc(-z / sqrt 2) / 2 in long double for u <= 1/2 and by
//         Phi^-1(u) = -Phi^-1(1 - u) above (1 - u is exact).
//     Gaussian and lognormal values are computed in long double from the
//     exact u1, u2 and returned rounded to double: this is the FP64 oracle
//     the tolerances |gpu - oracle| <= 2e-6 max(1,|x|) (FP32) and
//     1e-14 max(1,|x|) (FP64) are stated against.
//
// Pins (tests/test_oracle_*.py): Philox blocks equal Triton's independent
// Philox4x32-10; MRG32k3a has full-period transition matrices (orders checked
// against sympy's primitivity test), jumps equal stepping, powers compose;
// conversions equal exact rationals; Box-Muller matches closed forms and the
// normal / lognormal laws.  The sign of the MRG32k3a output combination
// z = x1 - x2 (both signs give statistically identical streams, so no CPU
// pin sees it) is pinned on the GPU against cuRAND's independent MRG32k3a,
// driven as a black box (tests/test_gpu_curand_pin.py), which also checks the
// Philox blocks a second time.  tests/test_oracle_planted.py plants 28
// plausible single mistakes in copies of this file; each fails a CPU pin.
//
// Built with -O2 -ffp-contract=off so that no multiply-add is contracted.

#include <cmath>
#include <cstdint>
#include <cstring>

namespace {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of a 4x32-bit S-P
// network; each round multiplies counter words 0 and 2 by two fixed
// constants, swaps the halves and mixes in the round key; the key is bumped
// by two Weyl constants between rounds.
const uint32_t PHILOX_M0 = 0xD2511F53u;  // multiplies counter word 0
const uint32_t PHILOX_M1 = 0xCD9E8D57u;  // multiplies counter word 2
const uint32_t PHILOX_W0 = 0x9E3779B9u;  // key bump, key word 0
const uint32_t PHILOX_W1 = 0xBB67AE85u;  // key bump, key word 1

void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += PHILOX_W0;
      k[1] += PHILOX_W1;
    }
    philox_round(c, k);
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Word g of the Philox stream for a given seed.
uint32_t philox_word(uint64_t seed, u128 g) {
  u128 block = g >> 2;
  uint32_t ctr[4];
  for (int i = 0; i < 4; ++i) ctr[i] = (uint32_t)(block >> (32 * i));
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  philox4x32_10(ctr, key, out);
  return out[(unsigned)(g & 3)];
}

// ---------------------------------------------------------------- MRG32k3a
// L'Ecuyer (1999), combined multiple recursive generator:
//   x1_n = (a12 x1_{n-2} - a13 x1_{n-3}) mod m1
//   x2_n = (a21 x2_{n-1} - a23 x2_{n-3}) mod m2
//   z_n  = (x1_n - x2_n) mod m1
const int64_t MRG_M1 = 4294967087LL;  // 2^32 - 209
const int64_t MRG_M2 = 4294944443LL;  // 2^32 - 22853
const int64_t MRG_A12 = 1403580;
const int64_t MRG_A13 = 810728;
const int64_t MRG_A21 = 527612;
const int64_t MRG_A23 = 1370589;

struct MrgState {
  // x1[0..2] = (x1_{n-3}, x1_{n-2}, x1_{n-1}); same for x2.
  int64_t x1[3];
  int64_t x2[3];
};

int64_t mod_floor(int64_t v, int64_t m) {
  int64_t r = v % m;
  return r < 0 ? r + m : r;
}

MrgState mrg_seed(uint64_t seed) {
  MrgState s;
  s.x1[0] = 1;
  s.x1[1] = 1;
  s.x1[2] = (int64_t)(seed % (uint64_t)MRG_M1);
  s.x2[0] = 1;
  s.x2[1] = 1;
  s.x2[2] = 1;
  return s;
}

// One step of the recursion; returns the output word z_n.
uint32_t mrg_step(MrgState& s) {
  int64_t n1 = mod_floor(MRG_A12 * s.x1[1] - MRG_A13 * s.x1[0], MRG_M1);
  int64_t n2 = mod_floor(MRG_A21 * s.x2[2] - MRG_A23 * s.x2[0], MRG_M2);
  s.x1[0] = s.x1[1]; s.x1[1] = s.x1[2]; s.x1[2] = n1;
  s.x2[0] = s.x2[1]; s.x2[1] = s.x2[2]; s.x2[2] = n2;
  return (uint32_t)mod_floor(n1 - n2, MRG_M1);
}

// 3x3 matrices mod m acting on the column vector (x_{n-3}, x_{n-2}, x_{n-1}).
struct Mat3 {
  uint64_t a[3][3];
};

uint64_t mulmod(uint64_t x, uint64_t y, uint64_t m) {
  return (uint64_t)(((u128)x * (u128)y) % (u128)m);
}

Mat3 mat_mul(const Mat3& A, const Mat3& B, uint64_t m) {
  Mat3 C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      uint64_t acc = 0;
      for (int k = 0; k < 3; ++k) acc = (acc + mulmod(A.a[i][k], B.a[k][j], m)) % m;
      C.a[i][j] = acc;
    }
  return C;
}

Mat3 mat_identity() {
  Mat3 I;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) I.a[i][j] = (i == j) ? 1 : 0;
  return I;
}

// The one-step transition matrix of component 1 or 2 (companion form).
Mat3 mrg_transition(int comp) {
  Mat3 A;
  std::memset(&A, 0, sizeof(A));
  A.a[0][1] = 1;  // new x_{n-3} = old x_{n-2}
  A.a[1][2] = 1;  // new x_{n-2} = old x_{n-1}
  if (comp == 1) {
    A.a[2][0] = (uint64_t)(MRG_M1 - MRG_A13);
    A.a[2][1] = (uint64_t)MRG_A12;
    A.a[2][2] = 0;
  } else {
    A.a[2][0] = (uint64_t)(MRG_M2 - MRG_A23);
    A.a[2][1] = 0;
    A.a[2][2] = (uint64_t)MRG_A21;
  }
  return A;
}

// A^e mod m by square-and-multiply over the bits of a little-endian exponent.
Mat3 mat_pow_bytes(int comp, const uint8_t* e, int nbytes) {
  uint64_t m = (comp == 1) ? (uint64_t)MRG_M1 : (uint64_t)MRG_M2;
  Mat3 result = mat_identity();
  Mat3 base = mrg_transition(comp);
  for (int byte = 0; byte < nbytes; ++byte)
    for (int bit = 0; bit < 8; ++bit) {
      if ((e[byte] >> bit) & 1) result = mat_mul(result, base, m);
      base = mat_mul(base, base, m);
    }
  return result;
}

Mat3 mat_pow128(int comp, u128 e) {
  uint8_t bytes[16];
  for (int i = 0; i < 16; ++i) bytes[i] = (uint8_t)(e >> (8 * i));
  return mat_pow_bytes(comp, bytes, 16);
}

void mat_apply(const Mat3& A, int64_t x[3], uint64_t m) {
  uint64_t y[3];
  for (int i = 0; i < 3; ++i) {
    uint64_t acc = 0;
    for (int k = 0; k < 3; ++k) acc = (acc + mulmod(A.a[i][k], (uint64_t)x[k], m)) % m;
    y[i] = acc;
  }
  for (int i = 0; i < 3; ++i) x[i] = (int64_t)y[i];
}

// State after skipping k steps from s.
void mrg_skip(MrgState& s, u128 k) {
  Mat3 A1 = mat_pow128(1, k);
  Mat3 A2 = mat_pow128(2, k);
  mat_apply(A1, s.x1, (uint64_t)MRG_M1);
  mat_apply(A2, s.x2, (uint64_t)MRG_M2);
}

// ---------------------------------------------------------------- words
enum { ENGINE_PHILOX = 0, ENGINE_MRG = 1 };
enum {
  DIST_BITS = 0,
  DIST_UNIFORM = 1,
  DIST_GAUSSIAN = 2,
  DIST_LOGNORMAL = 3,
  DIST_GAUSSIAN_ICDF = 4,
  DIST_LOGNORMAL_ICDF = 5
};
enum { DT_U32 = 0, DT_F32 = 1, DT_F64 = 2 };

u128 make_u128(uint64_t lo, uint64_t hi) { return ((u128)hi << 64) | (u128)lo; }

// Words [off, off + n) of the engine's stream, in order.
void engine_words(int engine, uint64_t seed, u128 off, int64_t n, uint32_t* out) {
  if (engine == ENGINE_PHILOX) {
    for (int64_t i = 0; i < n; ++i) out[i] = philox_word(seed, off + (u128)i);
  } else {
    MrgState s = mrg_seed(seed);
    mrg_skip(s, off);
    for (int64_t i = 0; i < n; ++i) out[i] = mrg_step(s);
  }
}

// ---------------------------------------------------------------- transforms
// Exact word -> uniform conversions (the values are exactly representable).
float u01_f32(uint32_t w) { return (float)std::ldexp((double)(w >> 8), -24); }
float u01_f32_open0(uint32_t w) { return (float)std::ldexp((double)((w >> 8) + 1u), -24); }

double u01_f64(uint32_t wa, uint32_t wb) {
  uint64_t x = (((uint64_t)wa << 32) | (uint64_t)wb) >> 11;
  return std::ldexp((double)x, -53);
}
double u01_f64_open0(uint32_t wa, uint32_t wb) {
  uint64_t x = (((uint64_t)wa << 32) | (uint64_t)wb) >> 11;
  return std::ldexp((double)(x + 1u), -53);
}

// Range transform of Sec. 4.3, Listing 2, made exact: each operation is a
// separate rounded float operation (the file is compiled without
// contraction), and a result that rounds up to b is moved below b.
float range_f32(float u, float a, float b) {
  float d = b - a;
  float t = d * u;
  float r = a + t;
  if (r >= b) r = std::nextafter(b, a);
  return r;
}
double range_f64(double u, double a, double b) {
  double d = b - a;
  double t = d * u;
  double r = a + t;
  if (r >= b) r = std::nextafter(b, a);
  return r;
}

const long double PI_L = 3.141592653589793238462643383279502884L;

// Box-Muller on exact u1 in (0,1], u2 in [0,1), in long double.
void box_muller_ld(long double u1, long double u2, long double* z0, long double* z1) {
  long double rho = std::sqrt(-2.0L * std::log(u1));
  long double ang = 2.0L * PI_L * u2;
  *z0 = rho * std::cos(ang);
  *z1 = rho * std::sin(ang);
}

// ---------------------------------------------------------------- ICDF
// Inverse-CDF method (oneMKL's icdf method of its gaussian / lognormal
// distributions, Sec. 4.1): z = Phi^-1(u) for one open-interval uniform per
// output.  Reading: u = (k + 1/2) 2^-23 with k = w >> 9 (FP32) and
// u = (x + 1/2) 2^-52 with x = ((w_a << 32 | w_b) >> 12) (FP64), exact
// midpoints in (0, 1) symmetric about 1/2.
float u_mid_f32(uint32_t w) { return (float)std::ldexp(2.0 * (double)(w >> 9) + 1.0, -24); }
double u_mid_f64(uint32_t wa, uint32_t wb) {
  uint64_t x = (((uint64_t)wa << 32) | (uint64_t)wb) >> 12;
  return std::ldexp(2.0 * (double)x + 1.0, -53);
}

// Phi(z) = erfc(-z / sqrt 2) / 2 in long double.
long double phi_ld(long double z) {
  const long double SQRT1_2 = 0.707106781186547524400844362104849039L;
  return 0.5L * std::erfc(-z * SQRT1_2);
}

// Phi^-1(u) by bisection on Phi (monotone), then Newton steps; plain and slow.
// Only called for u <= 1/2, where Phi(z) = erfc(-z / sqrt 2) / 2 keeps full
// relative precision; the upper half uses Phi^-1(u) = -Phi^-1(1 - u) with
// 1 - u exact (see icdf_z).
long double inv_phi_lower(long double u) {
  long double lo = -40.0L, hi = 40.0L;
  for (int it = 0; it < 200; ++it) {  // bisection to a tight bracket
    long double mid = 0.5L * (lo + hi);
    if (phi_ld(mid) < u) lo = mid; else hi = mid;
    if (hi - lo < 1e-12L) break;
  }
  long double z = 0.5L * (lo + hi);
  const long double INV_SQRT_2PI = 0.398942280401432677939946059934381868L;
  for (int it = 0; it < 4; ++it) {  // Newton: z -= (Phi(z) - u) / phi(z)
    long double dens = INV_SQRT_2PI * std::exp(-0.5L * z * z);
    z -= (phi_ld(z) - u) / dens;
  }
  return z;
}

// z = Phi^-1(u) for an exact midpoint u in (0, 1).
long double icdf_z(long double u) {
  return u <= 0.5L ? inv_phi_lower(u) : -inv_phi_lower(1.0L - u);
}

int words_per_output(int dtype) { return dtype == DT_F64 ? 2 : 1; }

bool is_pair_dist(int dist) { return dist == DIST_GAUSSIAN || dist == DIST_LOGNORMAL; }

// Words consumed by n outputs (a Box-Muller pair is always consumed whole).
uint64_t words_for(int dist, int dtype, int64_t n) {
  uint64_t wpo = (uint64_t)words_per_output(dtype);
  uint64_t un = (uint64_t)n;
  if (is_pair_dist(dist)) un = (un + 1u) / 2u * 2u;
  return un * wpo;
}

bool valid_combo(int dist, int dtype) {
  if (dist == DIST_BITS) return dtype == DT_U32;
  if (dist == DIST_UNIFORM || dist == DIST_GAUSSIAN || dist == DIST_LOGNORMAL ||
      dist == DIST_GAUSSIAN_ICDF || dist == DIST_LOGNORMAL_ICDF)
    return dtype == DT_F32 || dtype == DT_F64;
  return false;
}

// Applies the distribution to a word sequence that starts at a pair boundary.
// out: U32 bits -> uint32[n]; uniform F32 -> float[n]; uniform F64 -> double[n];
// gaussian / lognormal (either dtype) -> double[n] holding the long double
// result rounded to double.
void transform_words(int dist, int dtype, double p0, double p1, int64_t n,
                     const uint32_t* w, void* out) {
  if (dist == DIST_BITS) {
    uint32_t* o = (uint32_t*)out;
    for (int64_t i = 0; i < n; ++i) o[i] = w[i];
    return;
  }
  if (dist == DIST_UNIFORM) {
    if (dtype == DT_F32) {
      float* o = (float*)out;
      float a = (float)p0, b = (float)p1;
      for (int64_t i = 0; i < n; ++i) o[i] = range_f32(u01_f32(w[i]), a, b);
    } else {
      double* o = (double*)out;
      for (int64_t i = 0; i < n; ++i) o[i] = range_f64(u01_f64(w[2 * i], w[2 * i + 1]), p0, p1);
    }
    return;
  }
  if (dist == DIST_GAUSSIAN_ICDF || dist == DIST_LOGNORMAL_ICDF) {
    double* o = (double*)out;
    long double mean, sd;
    if (dtype == DT_F32) {
      mean = (long double)(float)p0;
      sd = (long double)(float)p1;
    } else {
      mean = (long double)p0;
      sd = (long double)p1;
    }
    for (int64_t i = 0; i < n; ++i) {
      long double u = dtype == DT_F32 ? (long double)u_mid_f32(w[i])
                                      : (long double)u_mid_f64(w[2 * i], w[2 * i + 1]);
      long double v = mean + sd * icdf_z(u);
      if (dist == DIST_LOGNORMAL_ICDF) v = std::exp(v);
      o[i] = (double)v;
    }
    return;
  }
  // Box-Muller family.
  double* o = (double*)out;
  long double mean, sd;
  if (dtype == DT_F32) {
    mean = (long double)(float)p0;
    sd = (long double)(float)p1;
  } else {
    mean = (long double)p0;
    sd = (long double)p1;
  }
  int64_t pairs = (n + 1) / 2;
  for (int64_t k = 0; k < pairs; ++k) {
    long double u1, u2;
    if (dtype == DT_F32) {
      u1 = (long double)u01_f32_open0(w[2 * k]);
      u2 = (long double)u01_f32(w[2 * k + 1]);
    } else {
      u1 = (long double)u01_f64_open0(w[4 * k], w[4 * k + 1]);
      u2 = (long double)u01_f64(w[4 * k + 2], w[4 * k + 3]);
    }
    long double z[2];
    box_muller_ld(u1, u2, &z[0], &z[1]);
    for (int j = 0; j < 2; ++j) {
      int64_t i = 2 * k + j;
      if (i >= n) break;
      long double v = mean + sd * z[j];
      if (dist == DIST_LOGNORMAL) v = std::exp(v);
      o[i] = (double)v;
    }
  }
}

}  // namespace

extern "C" {

// One Philox4x32-10 block: out = Philox(ctr, key).
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

// Words [off, off + n) of engine `engine` (0 Philox, 1 MRG32k3a) seeded with
// `seed`; off is the 128-bit word offset (off_lo + 2^64 off_hi).
int oracle_words(int engine, uint64_t seed, uint64_t off_lo, uint64_t off_hi, int64_t n,
                 uint32_t* out) {
  if (n < 0 || (engine != ENGINE_PHILOX && engine != ENGINE_MRG)) return 1;
  engine_words(engine, seed, make_u128(off_lo, off_hi), n, out);
  return 0;
}

// MRG32k3a seeded state as six values (x1_{-3}, x1_{-2}, x1_{-1}, x2_{-3}, x2_{-2}, x2_{-1}).
void oracle_mrg_seed_state(uint64_t seed, uint64_t* st) {
  MrgState s = mrg_seed(seed);
  for (int i = 0; i < 3; ++i) {
    st[i] = (uint64_t)s.x1[i];
    st[3 + i] = (uint64_t)s.x2[i];
  }
}

// Advances a six-value state by one step; returns the output word.
uint32_t oracle_mrg_step(uint64_t* st) {
  MrgState s;
  for (int i = 0; i < 3; ++i) {
    s.x1[i] = (int64_t)st[i];
    s.x2[i] = (int64_t)st[3 + i];
  }
  uint32_t z = mrg_step(s);
  for (int i = 0; i < 3; ++i) {
    st[i] = (uint64_t)s.x1[i];
    st[3 + i] = (uint64_t)s.x2[i];
  }
  return z;
}

// Advances a six-value state by k = k_lo + 2^64 k_hi steps through matrix powers.
void oracle_mrg_skip(uint64_t* st, uint64_t k_lo, uint64_t k_hi) {
  MrgState s;
  for (int i = 0; i < 3; ++i) {
    s.x1[i] = (int64_t)st[i];
    s.x2[i] = (int64_t)st[3 + i];
  }
  mrg_skip(s, make_u128(k_lo, k_hi));
  for (int i = 0; i < 3; ++i) {
    st[i] = (uint64_t)s.x1[i];
    st[3 + i] = (uint64_t)s.x2[i];
  }
}

// A_comp^e mod m_comp (row-major, 9 values) for a little-endian exponent of
// nbytes bytes (comp = 1 or 2).
int oracle_mrg_matrix_power(int comp, const uint8_t* e, int nbytes, uint64_t* out9) {
  if (comp != 1 && comp != 2) return 1;
  Mat3 A = mat_pow_bytes(comp, e, nbytes);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out9[3 * i + j] = A.a[i][j];
  return 0;
}

uint64_t oracle_words_for(int dist, int dtype, int64_t n) { return words_for(dist, dtype, n); }

// Exact conversions, exposed for the special-case tests.
float oracle_u01_f32(uint32_t w) { return u01_f32(w); }
double oracle_u01_f64(uint32_t wa, uint32_t wb) { return u01_f64(wa, wb); }
float oracle_uniform_f32(uint32_t w, float a, float b) { return range_f32(u01_f32(w), a, b); }
double oracle_uniform_f64(uint32_t wa, uint32_t wb, double a, double b) {
  return range_f64(u01_f64(wa, wb), a, b);
}

// Applies a distribution to n outputs' worth of given words (see transform_words).
int oracle_transform_words(int dist, int dtype, double p0, double p1, int64_t n,
                           const uint32_t* words, void* out) {
  if (n < 0 || !valid_combo(dist, dtype)) return 1;
  transform_words(dist, dtype, p0, p1, n, words, out);
  return 0;
}

// The whole path: n outputs of distribution (dist, dtype, p0, p1) from the
// engine's words starting at word offset off.  Output layout as in
// transform_words.  Returns 0 on success, 1 on an invalid argument.
int oracle_generate(int engine, uint64_t seed, uint64_t off_lo, uint64_t off_hi, int dist,
                    int dtype, double p0, double p1, int64_t n, void* out) {
  if (n < 0 || !valid_combo(dist, dtype)) return 1;
  if (engine != ENGINE_PHILOX && engine != ENGINE_MRG) return 1;
  uint64_t nw = words_for(dist, dtype, n);
  uint32_t* w = new uint32_t[nw > 0 ? nw : 1];
  engine_words(engine, seed, make_u128(off_lo, off_hi), (int64_t)nw, w);
  transform_words(dist, dtype, p0, p1, n, w, out);
  delete[] w;
  return 0;
}

// The whole path for an engine seeded by a list of 1..6 32-bit words
// (oneMKL's seed initializer lists, Sec. 4.1).  Reading: Philox key = words
// 0, 1 and starting block counter = words 2..5 (word offset 4 counter + off);
// MRG32k3a x1_{-1}, x1_{-2}, x1_{-3} = words 0..2 (mod m1) and x2_{-1},
// x2_{-2}, x2_{-3} = words 3..5 (mod m2), missing words 1.
int oracle_generate_words(int engine, const uint32_t* words, int count, uint64_t off_lo,
                          uint64_t off_hi, int dist, int dtype, double p0, double p1, int64_t n,
                          void* out) {
  if (n < 0 || count < 1 || count > 6 || !valid_combo(dist, dtype)) return 1;
  uint32_t w[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < count; ++i) w[i] = words[i];
  const u128 off = make_u128(off_lo, off_hi);
  const uint64_t nw = words_for(dist, dtype, n);
  uint32_t* buf = new uint32_t[nw > 0 ? nw : 1];
  if (engine == ENGINE_PHILOX) {
    const uint64_t seed = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    u128 counter = 0;
    for (int i = 0; i < 4; ++i) counter |= (u128)w[2 + i] << (32 * i);
    const u128 start = counter * 4 + off;
    for (uint64_t i = 0; i < nw; ++i) buf[i] = philox_word(seed, start + (u128)i);
  } else if (engine == ENGINE_MRG) {
    MrgState st;
    for (int i = 0; i < 3; ++i) {
      st.x1[2 - i] = i < count ? (int64_t)(w[i] % (uint32_t)MRG_M1) : 1;
      st.x2[2 - i] = 3 + i < count ? (int64_t)(w[3 + i] % (uint32_t)MRG_M2) : 1;
    }
    mrg_skip(st, off);
    for (uint64_t i = 0; i < nw; ++i) buf[i] = mrg_step(st);
  } else {
    delete[] buf;
    return 1;
  }
  transform_words(dist, dtype, p0, p1, n, buf, out);
  delete[] buf;
  return 0;
}

}  // extern "C"
