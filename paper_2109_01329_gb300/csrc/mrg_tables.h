// MRG32k3a constants and the compile-time table of transition-matrix powers
// A1^(2^j) mod m1 and A2^(2^j) mod m2, j = 0..127, used for skip-ahead on
// both the host (engine offsets) and the device (per-thread jumps).
//
// MRG32k3a (L'Ecuyer 1999) is the "MRG-based generator" family the paper's
// library offers beside Philox (Sec. 4.1).  State vectors are
// (x_{n-3}, x_{n-2}, x_{n-1}); one step is multiplication by the companion
// matrix A of the recursion.  A jump by k steps multiplies by A^k, built from
// the binary expansion of k with the powers A^(2^j) tabulated here.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define GRNG_HD __host__ __device__
#else
#define GRNG_HD
#endif

namespace grng {
namespace mrg {

constexpr uint32_t M1 = 4294967087u;  // 2^32 - 209
constexpr uint32_t M2 = 4294944443u;  // 2^32 - 22853
constexpr uint32_t C1 = 209u;         // 2^32 mod m1
constexpr uint32_t C2 = 22853u;       // 2^32 mod m2
constexpr uint32_t A12 = 1403580u;
constexpr uint32_t A13 = 810728u;
constexpr uint32_t A21 = 527612u;
constexpr uint32_t A23 = 1370589u;

constexpr int kLevels = 128;

// pow2[c][j] = A_{c+1}^(2^j), row-major 3x3.
struct PowTable {
  uint32_t m[2][kLevels][9];
};

constexpr uint32_t cx_mulmod(uint32_t a, uint32_t b, uint32_t m) {
  return (uint32_t)(((uint64_t)a * (uint64_t)b) % (uint64_t)m);
}

constexpr void cx_matsq(const uint32_t* a, uint32_t* out, uint32_t m) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      uint64_t acc = 0;
      for (int k = 0; k < 3; ++k) acc = (acc + cx_mulmod(a[3 * i + k], a[3 * k + j], m)) % m;
      out[3 * i + j] = (uint32_t)acc;
    }
}

constexpr PowTable make_pow_table() {
  PowTable t{};
  // A1: new x_{n-1} = a12 x_{n-2} - a13 x_{n-3}; A2: a21 x_{n-1} - a23 x_{n-3}.
  const uint32_t a1[9] = {0, 1, 0, 0, 0, 1, M1 - A13, A12, 0};
  const uint32_t a2[9] = {0, 1, 0, 0, 0, 1, M2 - A23, 0, A21};
  for (int i = 0; i < 9; ++i) {
    t.m[0][0][i] = a1[i];
    t.m[1][0][i] = a2[i];
  }
  for (int j = 1; j < kLevels; ++j) {
    cx_matsq(t.m[0][j - 1], t.m[0][j], M1);
    cx_matsq(t.m[1][j - 1], t.m[1][j], M2);
  }
  return t;
}

// (hi * 2^32 + lo) mod m for m = 2^32 - c, any 64-bit value.
GRNG_HD inline uint32_t reduce64(uint64_t p, uint32_t m, uint32_t c) {
  uint64_t t = (p & 0xFFFFFFFFull) + (p >> 32) * (uint64_t)c;  // < 2^32 + 2^32 c
  t = (t & 0xFFFFFFFFull) + (t >> 32) * (uint64_t)c;           // < 2^32 + 2^16 c
  t = (t & 0xFFFFFFFFull) + (t >> 32) * (uint64_t)c;           // < 2^32 + c
  return (uint32_t)(t >= m ? t - m : t);
}

// y = M x mod m for a 3x3 matrix and 3-vector of residues.
GRNG_HD inline void matvec(const uint32_t* M, uint32_t* x, uint32_t m, uint32_t c) {
  uint32_t y[3];
  for (int i = 0; i < 3; ++i) {
    uint64_t acc = 0;
    for (int k = 0; k < 3; ++k) acc += reduce64((uint64_t)M[3 * i + k] * x[k], m, c);
    y[i] = reduce64(acc, m, c);
  }
  x[0] = y[0];
  x[1] = y[1];
  x[2] = y[2];
}

}  // namespace mrg
}  // namespace grng
