// Host side of the C ABI declared in include/grng.h: engines (seed, 128-bit
// word offset, cached MRG32k3a state), argument checks, the choice of kernel
// variant, offset bookkeeping and the chunked generate-to-host flow.
//
// The engine object mirrors the generator of the paper's native flow
// (Sec. 4.2: create, set seed and offset, generate, destroy) and oneMKL's
// engine classes (Sec. 4.1), whose sequences continue across generate calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "grng.h"
#include "grng_internal.h"
#include "bm64_fixed.cuh"
#include "mrg_tables.h"

struct grng_engine {
  int32_t kind;
  uint64_t seed;            // single seed, or the Philox key of a word seed
  uint32_t nwords;          // 0: seeded by `seed`; 1..6: by words[]
  uint32_t words[6];
  uint64_t off_lo, off_hi;  // 128-bit word offset
  uint32_t mrg[6];          // MRG32k3a: state at the current offset
};

namespace grng {
namespace {

thread_local char g_last_error[512] = "";

constexpr mrg::PowTable kHostPow = mrg::make_pow_table();

// Applies A^(e_lo + 2^64 e_hi) to an MRG32k3a state (x1[3], x2[3]).
void mrg_jump_host(uint32_t* st, uint64_t e_lo, uint64_t e_hi) {
  for (int j = 0; j < 128; ++j) {
    const uint64_t word = j < 64 ? e_lo : e_hi;
    if ((word >> (j & 63)) & 1u) {
      mrg::matvec(kHostPow.m[0][j], st, mrg::M1, mrg::C1);
      mrg::matvec(kHostPow.m[1][j], st + 3, mrg::M2, mrg::C2);
    }
  }
}

void mrg_seed_state(uint64_t seed, uint32_t* st) {
  st[0] = 1;
  st[1] = 1;
  st[2] = (uint32_t)(seed % (uint64_t)mrg::M1);
  st[3] = 1;
  st[4] = 1;
  st[5] = 1;
}

// MRG32k3a state from seed words: words 0..2 are x1_{-1}, x1_{-2}, x1_{-3}
// (mod m1), words 3..5 the same for x2 (mod m2); missing words are 1, so one
// word w gives the single-seed state (1, 1, w mod m1), (1, 1, 1).
void mrg_words_state(const uint32_t* w, uint32_t n, uint32_t* st) {
  for (int i = 0; i < 3; ++i) {
    st[2 - i] = i < (int)n ? w[i] % mrg::M1 : 1u;
    st[5 - i] = 3 + i < (int)n ? w[3 + i] % mrg::M2 : 1u;
  }
}

void init_engine(grng_engine* e, int32_t kind, uint64_t seed, uint64_t off_lo, uint64_t off_hi) {
  e->kind = kind;
  e->seed = seed;
  e->off_lo = off_lo;
  e->off_hi = off_hi;
  std::memset(e->mrg, 0, sizeof(e->mrg));
  if (kind == GRNG_MRG32K3A) {
    if (e->nwords > 0) {
      mrg_words_state(e->words, e->nwords, e->mrg);
    } else {
      mrg_seed_state(seed, e->mrg);
    }
    mrg_jump_host(e->mrg, off_lo, off_hi);
  }
}

// Offsets are taken mod 2^128.  The cached MRG32k3a state is always the
// state at that reduced offset: an advance that wraps recomputes it from the
// seed (within one call a fill that crosses 2^128 continues the recursion).
void advance_engine(grng_engine* e, uint64_t n_lo, uint64_t n_hi) {
  const uint64_t lo = e->off_lo + n_lo;
  const uint64_t c0 = (lo < e->off_lo) ? 1u : 0u;
  const uint64_t hi1 = e->off_hi + n_hi;
  const bool wrapped = hi1 < e->off_hi || (hi1 + c0) < hi1;
  e->off_hi = hi1 + c0;
  e->off_lo = lo;
  if (e->kind == GRNG_MRG32K3A) {
    if (wrapped) {
      init_engine(e, e->kind, e->seed, e->off_lo, e->off_hi);
    } else {
      mrg_jump_host(e->mrg, n_lo, n_hi);
    }
  }
}

bool is_pair_dist(int32_t kind) { return kind == GRNG_GAUSSIAN || kind == GRNG_LOGNORMAL; }

constexpr int64_t kMaxElements = int64_t(1) << 40;

grng_status check_dist(const grng_distribution* d) {
  if (d == nullptr) {
    set_error("distribution is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  const bool dt_float = d->dtype == GRNG_F32 || d->dtype == GRNG_F64;
  switch (d->kind) {
    case GRNG_BITS:
      if (d->dtype != GRNG_U32) {
        set_error("bits distribution needs dtype U32");
        return GRNG_ERR_INVALID_ARG;
      }
      return GRNG_OK;
    case GRNG_UNIFORM: {
      if (!dt_float) {
        set_error("uniform needs dtype F32 or F64");
        return GRNG_ERR_INVALID_ARG;
      }
      if (d->dtype == GRNG_F32) {
        const float a = (float)d->p0, b = (float)d->p1;
        const float w = b - a;
        if (!std::isfinite(a) || !std::isfinite(b) || !(a < b) || !std::isfinite(w)) {
          set_error("uniform F32 needs finite a < b with b - a finite in float");
          return GRNG_ERR_INVALID_ARG;
        }
      } else {
        const double a = d->p0, b = d->p1;
        if (!std::isfinite(a) || !std::isfinite(b) || !(a < b) || !std::isfinite(b - a)) {
          set_error("uniform F64 needs finite a < b with b - a finite");
          return GRNG_ERR_INVALID_ARG;
        }
      }
      return GRNG_OK;
    }
    case GRNG_GAUSSIAN:
    case GRNG_LOGNORMAL:
    case GRNG_GAUSSIAN_ICDF:
    case GRNG_LOGNORMAL_ICDF: {
      if (!dt_float) {
        set_error("gaussian / lognormal need dtype F32 or F64");
        return GRNG_ERR_INVALID_ARG;
      }
      double m = d->p0, s = d->p1;
      if (d->dtype == GRNG_F32) {
        m = (float)m;
        s = (float)s;
      }
      if (!std::isfinite(m) || !std::isfinite(s) || !(s > 0)) {
        set_error("gaussian / lognormal need a finite mean and a finite stddev > 0");
        return GRNG_ERR_INVALID_ARG;
      }
      return GRNG_OK;
    }
    default:
      set_error("unknown distribution kind %d", d->kind);
      return GRNG_ERR_INVALID_ARG;
  }
}

uint64_t words_for_checked(const grng_distribution* d, int64_t n) {
  uint64_t un = (uint64_t)n;
  if (is_pair_dist(d->kind)) un = (un + 1u) / 2u * 2u;
  return un * (d->dtype == GRNG_F64 ? 2u : 1u);
}

int elem_size(int32_t dtype) { return dtype == GRNG_F64 ? 8 : 4; }

// When a + (b - a) u is exact for every 53-bit u, returns true and the
// integer form r = (A + x) 2^e used by the integer-only F64 variant.  The
// result equals the rounded form bit for bit because no rounding happens.
bool exact_affine_f64(double a, double b, int64_t* A, int32_t* e) {
  const double d = b - a;
  int k = 0;
  const double frac = std::frexp(d, &k);  // d = frac 2^k, frac in [0.5, 1)
  if (frac != 0.5) return false;          // d must be a power of two, 2^(k-1)
  const int kk = k - 1;
  const int ex = kk - 53;                 // ulp of the result grid
  if (ex < -1000) return false;
  const double a_scaled = std::ldexp(a, -ex);
  if (!(std::fabs(a_scaled) <= 9007199254740992.0)) return false;  // 2^53
  if (a_scaled != std::trunc(a_scaled)) return false;
  const int64_t Ai = (int64_t)a_scaled;
  if (Ai > 0 || Ai < -(int64_t(1) << 53)) return false;  // |A + x| < 2^53 for x < 2^53
  if (std::ldexp((double)(Ai + (int64_t(1) << 53)), ex) != b) return false;  // a + d == b exactly
  *A = Ai;
  *e = ex;
  return true;
}

// The integer form of the F64 uniform's product d u (u = x 2^-53): d's
// 53-bit significand and exponent, when every nonzero product is a normal
// double; and the clamp as a threshold on x.  a + d u with its two roundings
// is non-decreasing in x, so r >= b holds exactly from the smallest such x on;
// the host evaluates the same two roundings (volatile: never fused).
void uniform_f64_consts(double a, double b, TransformParams* t) {
  const double d = t->dd;
  int k = 0;
  const double f = std::frexp(d, &k);  // d = f 2^k, f in [0.5, 1)
  if (std::isfinite(d) && d > 0.0 && k >= -960) {
    const uint64_t D = (uint64_t)std::ldexp(f, 53);  // [2^52, 2^53)
    t->rd_hi = (uint32_t)(D >> 32);
    t->rd_lo = (uint32_t)D;
    t->rd_exp = k - 53;
    t->r_int = 1;
  }
  auto reaches = [&](uint64_t x) {
    volatile double u = std::ldexp((double)x, -53);
    volatile double prod = d * u;
    volatile double r = a + prod;
    return r >= b;
  };
  const uint64_t top = (uint64_t(1) << 53) - 1;
  if (!reaches(top)) {
    t->r_xthr = uint64_t(1) << 53;
    return;
  }
  uint64_t lo = 0, hi = top;  // reaches(hi); the threshold is in (lo, hi] unless reaches(0)
  if (reaches(0)) {
    t->r_xthr = 0;
    return;
  }
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (reaches(mid)) {
      hi = mid;
    } else {
      lo = mid;
    }
  }
  t->r_xthr = hi;
}

int choose_variant(const grng_distribution* d, TransformParams* t) {
  std::memset(t, 0, sizeof(*t));
  switch (d->kind) {
    case GRNG_BITS: return V_BITS;
    case GRNG_UNIFORM:
      if (d->dtype == GRNG_F32) {
        const float a = (float)d->p0, b = (float)d->p1;
        t->fa = a;
        t->fb = b;
        t->fd = b - a;
        t->fbprev = std::nextafter(b, a);
        return (a == 0.0f && b == 1.0f) ? V_U01_F32 : V_UNI_F32;
      } else {
        const double a = d->p0, b = d->p1;
        t->da = a;
        t->db = b;
        t->dd = b - a;
        t->dbprev = std::nextafter(b, a);
        if (a == 0.0 && b == 1.0) return V_U01_F64;
        int64_t A = 0;
        int32_t e = 0;
        if (exact_affine_f64(a, b, &A, &e)) {
          t->aff_a = A;
          t->aff_exp = e;
          return V_AFF_F64;
        }
        uniform_f64_consts(a, b, t);
        return V_UNI_F64;
      }
    case GRNG_GAUSSIAN:
    case GRNG_LOGNORMAL: {
      const bool logn = d->kind == GRNG_LOGNORMAL;
      if (d->dtype == GRNG_F32) {
        t->fmean = (float)d->p0;
        t->fsd = (float)d->p1;
        return logn ? V_LOGN_F32 : V_GAUSS_F32;
      }
      t->dmean = d->p0;
      t->dsd = d->p1;
      if (logn) {
        uint64_t em = 0, sm = 0;
        int ee = 0, se = 0;
        t->ln_fast = bm64::lognormal_consts(d->p0, d->p1, em, ee, sm, se) ? 1 : 0;
        t->ln_em_mant = em;
        t->ln_em_exp = ee;
        t->ln_s_mant = sm;
        t->ln_s_exp = se;
        return V_LOGN_F64;
      }
      // fma(1, z, 0) == z, so (0, 1) drops the affine step exactly
      return (d->p0 == 0.0 && d->p1 == 1.0) ? V_STDGAUSS_F64 : V_GAUSS_F64;
    }
    case GRNG_GAUSSIAN_ICDF:
    case GRNG_LOGNORMAL_ICDF: {
      const bool logn = d->kind == GRNG_LOGNORMAL_ICDF;
      if (d->dtype == GRNG_F32) {
        t->fmean = (float)d->p0;
        t->fsd = (float)d->p1;
        return logn ? V_ICDF_LOGN_F32 : V_ICDF_GAUSS_F32;
      }
      t->dmean = d->p0;
      t->dsd = d->p1;
      if (logn) {
        uint64_t em = 0, sm = 0;
        int ee = 0, se = 0;
        t->ln_fast = bm64::lognormal_consts(d->p0, d->p1, em, ee, sm, se) ? 1 : 0;
        t->ln_em_mant = em;
        t->ln_em_exp = ee;
        t->ln_s_mant = sm;
        t->ln_s_exp = se;
      }
      return logn ? V_ICDF_LOGN_F64 : V_ICDF_GAUSS_F64;
    }
    default: return -1;
  }
}

grng_status fill(const grng_distribution* dist, grng_engine* e, int64_t n, int64_t num_streams,
                 uint64_t stride_lo, uint64_t stride_hi, void* dev_ptr, cudaStream_t stream) {
  FillRequest r;
  std::memset(&r, 0, sizeof(r));
  r.variant = choose_variant(dist, &r.t);
  r.engine_kind = e->kind;
  r.n = n;
  r.num_streams = num_streams;
  r.off_lo = e->off_lo;
  r.off_hi = e->off_hi;
  r.stride_lo = stride_lo;
  r.stride_hi = stride_hi;
  r.out = dev_ptr;
  r.key[0] = (uint32_t)e->seed;
  r.key[1] = (uint32_t)(e->seed >> 32);
  std::memcpy(r.mrg, e->mrg, sizeof(r.mrg));
  if (e->kind == GRNG_PHILOX4X32X10) return launch_philox(r, stream);
  return launch_mrg(r, stream);
}

grng_status check_ptr(const void* p, int64_t n, int32_t dtype) {
  if (n > 0 && p == nullptr) {
    set_error("output pointer is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  if (((uintptr_t)p % (uintptr_t)elem_size(dtype)) != 0) {
    set_error("output pointer is not aligned to its element size");
    return GRNG_ERR_INVALID_ARG;
  }
  return GRNG_OK;
}

std::mutex g_sms_mutex;
int g_sms[256];

// Copy stream and events for grng_generate_host, created once per device.
struct HostFlowState {
  bool ready = false;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t gen_done[2] = {nullptr, nullptr};
  cudaEvent_t copy_done[2] = {nullptr, nullptr};
  std::mutex mu;
};
HostFlowState g_host_flow[256];
std::mutex g_host_flow_init;

}  // namespace

grng_status fill_transform_params(const grng_distribution* d, TransformParams* t, int* variant) {
  const grng_status st = check_dist(d);
  if (st != GRNG_OK) return st;
  *variant = choose_variant(d, t);
  return GRNG_OK;
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int current_device_sms(int* device_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  if (device_out) *device_out = dev;
  if (dev < 0 || dev >= 256) return 1;
  std::lock_guard<std::mutex> g(g_sms_mutex);
  if (g_sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    g_sms[dev] = v;
  }
  return g_sms[dev];
}

}  // namespace grng

using namespace grng;

extern "C" {

const char* grng_status_string(grng_status s) {
  switch (s) {
    case GRNG_OK: return "GRNG_OK";
    case GRNG_ERR_INVALID_ARG: return "GRNG_ERR_INVALID_ARG";
    case GRNG_ERR_UNSUPPORTED: return "GRNG_ERR_UNSUPPORTED";
    case GRNG_ERR_OOM: return "GRNG_ERR_OOM";
    case GRNG_ERR_CUDA: return "GRNG_ERR_CUDA";
    case GRNG_ERR_TIMEOUT: return "GRNG_ERR_TIMEOUT";
    case GRNG_ERR_BUDGET: return "GRNG_ERR_BUDGET";
    default: return "GRNG_ERR_UNKNOWN";
  }
}

const char* grng_last_error(void) { return g_last_error; }

grng_status grng_engine_create_words(grng_engine_t* out, int32_t kind, const uint32_t* words,
                                     int32_t count, uint64_t offset) {
  if (out == nullptr || (count > 0 && words == nullptr) || count < 1 || count > 6) {
    set_error("out NULL, words NULL or count not in [1, 6]");
    return GRNG_ERR_INVALID_ARG;
  }
  if (kind != GRNG_PHILOX4X32X10 && kind != GRNG_MRG32K3A) {
    set_error("unknown engine kind %d", kind);
    return GRNG_ERR_INVALID_ARG;
  }
  uint32_t w[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < count; ++i) w[i] = words[i];
  uint64_t seed = 0, off_lo = offset, off_hi = 0;
  if (kind == GRNG_PHILOX4X32X10) {
    // key = words 0, 1; counter = words 2..5; word offset = 4 counter + offset
    seed = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    const uint64_t c_lo = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
    const uint64_t c_hi = (uint64_t)w[4] | ((uint64_t)w[5] << 32);
    const uint64_t b_lo = c_lo << 2, b_hi = (c_hi << 2) | (c_lo >> 62);
    off_lo = b_lo + offset;
    off_hi = b_hi + ((off_lo < b_lo) ? 1u : 0u);
  } else {
    uint32_t st[6];
    mrg_words_state(w, (uint32_t)count, st);
    if ((st[0] | st[1] | st[2]) == 0 || (st[3] | st[4] | st[5]) == 0) {
      set_error("an MRG32k3a component state of all zeros never leaves zero");
      return GRNG_ERR_INVALID_ARG;
    }
  }
  grng_engine* e = new (std::nothrow) grng_engine;
  if (e == nullptr) {
    set_error("engine allocation failed");
    return GRNG_ERR_OOM;
  }
  e->nwords = kind == GRNG_MRG32K3A ? (uint32_t)count : 0u;
  std::memcpy(e->words, w, sizeof(w));
  init_engine(e, kind, seed, off_lo, off_hi);
  *out = e;
  return GRNG_OK;
}

grng_status grng_engine_create(grng_engine_t* out, int32_t kind, uint64_t seed, uint64_t offset) {
  if (out == nullptr) {
    set_error("out is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  if (kind != GRNG_PHILOX4X32X10 && kind != GRNG_MRG32K3A) {
    set_error("unknown engine kind %d", kind);
    return GRNG_ERR_INVALID_ARG;
  }
  grng_engine* e = new (std::nothrow) grng_engine;
  if (e == nullptr) {
    set_error("engine allocation failed");
    return GRNG_ERR_OOM;
  }
  e->nwords = 0;
  std::memset(e->words, 0, sizeof(e->words));
  init_engine(e, kind, seed, offset, 0);
  *out = e;
  return GRNG_OK;
}

grng_status grng_engine_restore(grng_engine_t* out, const grng_engine_state* st) {
  if (out == nullptr || st == nullptr) {
    set_error("NULL argument");
    return GRNG_ERR_INVALID_ARG;
  }
  if (st->kind != GRNG_PHILOX4X32X10 && st->kind != GRNG_MRG32K3A) {
    set_error("unknown engine kind %d", st->kind);
    return GRNG_ERR_INVALID_ARG;
  }
  grng_engine* e = new (std::nothrow) grng_engine;
  if (e == nullptr) {
    set_error("engine allocation failed");
    return GRNG_ERR_OOM;
  }
  if (st->reserved > 6 || (st->reserved > 0 && st->kind != GRNG_MRG32K3A)) {
    delete e;
    set_error("state words: 0 (seed) or 1..6 for MRG32k3a");
    return GRNG_ERR_INVALID_ARG;
  }
  e->nwords = st->reserved;
  std::memcpy(e->words, st->words, sizeof(e->words));
  init_engine(e, st->kind, st->seed, st->offset_lo, st->offset_hi);
  *out = e;
  return GRNG_OK;
}

grng_status grng_engine_copy(grng_engine_t* out, grng_engine_t src) {
  if (out == nullptr || src == nullptr) {
    set_error("NULL argument");
    return GRNG_ERR_INVALID_ARG;
  }
  grng_engine* e = new (std::nothrow) grng_engine;
  if (e == nullptr) {
    set_error("engine allocation failed");
    return GRNG_ERR_OOM;
  }
  *e = *src;
  *out = e;
  return GRNG_OK;
}

grng_status grng_engine_skip_ahead(grng_engine_t e, uint64_t n_lo, uint64_t n_hi) {
  if (e == nullptr) {
    set_error("engine is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  advance_engine(e, n_lo, n_hi);
  return GRNG_OK;
}

grng_status grng_engine_get_state(grng_engine_t e, grng_engine_state* out) {
  if (e == nullptr || out == nullptr) {
    set_error("NULL argument");
    return GRNG_ERR_INVALID_ARG;
  }
  out->kind = e->kind;
  out->reserved = e->nwords;
  std::memcpy(out->words, e->words, sizeof(out->words));
  out->seed = e->seed;
  out->offset_lo = e->off_lo;
  out->offset_hi = e->off_hi;
  return GRNG_OK;
}

grng_status grng_engine_destroy(grng_engine_t e) {
  delete e;
  return GRNG_OK;
}

grng_status grng_words_for(const grng_distribution* dist, int64_t n, uint64_t* words_out) {
  grng_status st = check_dist(dist);
  if (st != GRNG_OK) return st;
  if (words_out == nullptr || n < 0) {
    set_error("words_out is NULL or n < 0");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n > kMaxElements) {
    set_error("n above 2^40");
    return GRNG_ERR_UNSUPPORTED;
  }
  *words_out = words_for_checked(dist, n);
  return GRNG_OK;
}

grng_status grng_generate(const grng_distribution* dist, grng_engine_t engine, int64_t n,
                          void* dev_ptr, grng_stream_t stream) {
  grng_status st = check_dist(dist);
  if (st != GRNG_OK) return st;
  if (engine == nullptr) {
    set_error("engine is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n < 0) {
    set_error("n < 0");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n > kMaxElements) {
    set_error("n above 2^40");
    return GRNG_ERR_UNSUPPORTED;
  }
  st = check_ptr(dev_ptr, n, dist->dtype);
  if (st != GRNG_OK) return st;
  if (n == 0) return GRNG_OK;
  st = fill(dist, engine, n, 1, 0, 0, dev_ptr, (cudaStream_t)stream);
  if (st != GRNG_OK) return st;
  advance_engine(engine, words_for_checked(dist, n), 0);
  return GRNG_OK;
}

grng_status grng_transform_words(const grng_distribution* dist, const uint32_t* dev_words,
                                 int64_t n, void* dev_out, grng_stream_t stream) {
  grng_status st = check_dist(dist);
  if (st != GRNG_OK) return st;
  if (n < 0) {
    set_error("n < 0");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n > kMaxElements) {
    set_error("n above 2^40");
    return GRNG_ERR_UNSUPPORTED;
  }
  st = check_ptr(dev_out, n, dist->dtype);
  if (st != GRNG_OK) return st;
  if (n > 0 && (dev_words == nullptr || ((uintptr_t)dev_words & 3u) != 0)) {
    set_error("words pointer is NULL or not 4-byte aligned");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n == 0) return GRNG_OK;
  TransformParams t;
  const int v = choose_variant(dist, &t);
  return launch_transform(v, t, dev_words, n, dev_out, (cudaStream_t)stream);
}

grng_status grng_generate_substreams(const grng_distribution* dist, grng_engine_t engine,
                                     int64_t n_per_stream, int64_t num_streams,
                                     uint64_t stride_lo, uint64_t stride_hi, void* dev_ptr,
                                     grng_stream_t stream) {
  grng_status st = check_dist(dist);
  if (st != GRNG_OK) return st;
  if (engine == nullptr) {
    set_error("engine is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n_per_stream < 0 || num_streams < 0) {
    set_error("negative size");
    return GRNG_ERR_INVALID_ARG;
  }
  if (num_streams > (int64_t(1) << 31) || n_per_stream > kMaxElements ||
      (num_streams > 0 && n_per_stream > kMaxElements / num_streams)) {
    set_error("num_streams * n_per_stream above 2^40 or num_streams above 2^31");
    return GRNG_ERR_UNSUPPORTED;
  }
  const int64_t total = n_per_stream * num_streams;
  st = check_ptr(dev_ptr, total, dist->dtype);
  if (st != GRNG_OK) return st;
  if (total == 0) return GRNG_OK;
  return fill(dist, engine, n_per_stream, num_streams, stride_lo, stride_hi, dev_ptr,
              (cudaStream_t)stream);
}

grng_status grng_generate_host(const grng_distribution* dist, grng_engine_t engine, int64_t n,
                               void* host_ptr, void* dev_work, size_t work_bytes,
                               grng_stream_t stream_in) {
  grng_status st = check_dist(dist);
  if (st != GRNG_OK) return st;
  if (engine == nullptr) {
    set_error("engine is NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n < 0) {
    set_error("n < 0");
    return GRNG_ERR_INVALID_ARG;
  }
  if (n > kMaxElements) {
    set_error("n above 2^40");
    return GRNG_ERR_UNSUPPORTED;
  }
  if (n == 0) return GRNG_OK;
  if (host_ptr == nullptr || dev_work == nullptr || work_bytes < (size_t(2) << 20) ||
      ((uintptr_t)dev_work & 255u) != 0) {
    set_error("host_ptr / dev_work NULL, dev_work not 256-byte aligned or under 2 MiB");
    return GRNG_ERR_INVALID_ARG;
  }
  const int es = elem_size(dist->dtype);
  // two halves; each chunk a multiple of 4 elements (whole pairs, 16-byte ends)
  const int64_t chunk = (int64_t)(work_bytes / 2 / (size_t)es) / 4 * 4;
  cudaStream_t stream = (cudaStream_t)stream_in;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    set_error("cudaGetDevice failed");
    return GRNG_ERR_CUDA;
  }
  HostFlowState& hs = g_host_flow[dev];
  {
    std::lock_guard<std::mutex> g(g_host_flow_init);
    if (!hs.ready) {
      bool ok = cudaStreamCreateWithFlags(&hs.copy_stream, cudaStreamNonBlocking) == cudaSuccess;
      for (int i = 0; i < 2 && ok; ++i) {
        ok = cudaEventCreateWithFlags(&hs.gen_done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&hs.copy_done[i], cudaEventDisableTiming) == cudaSuccess;
      }
      if (!ok) {
        set_error("creating the copy stream / events failed: %s",
                  cudaGetErrorString(cudaGetLastError()));
        return GRNG_ERR_CUDA;
      }
      hs.ready = true;
    }
  }
  std::lock_guard<std::mutex> flow_lock(hs.mu);
  grng_engine local = *engine;  // the engine commits only on success
  char* host = reinterpret_cast<char*>(host_ptr);
  char* work = reinterpret_cast<char*>(dev_work);
  int64_t done = 0;
  int64_t idx = 0;
  cudaError_t cerr = cudaSuccess;
  while (done < n) {
    const int h = (int)(idx & 1);
    const int64_t m = (n - done) < chunk ? (n - done) : chunk;
    char* half = work + (size_t)h * (size_t)chunk * (size_t)es;
    if (idx >= 2) {
      cerr = cudaStreamWaitEvent(stream, hs.copy_done[h], 0);
      if (cerr != cudaSuccess) break;
    }
    st = fill(dist, &local, m, 1, 0, 0, half, stream);
    if (st != GRNG_OK) break;
    advance_engine(&local, words_for_checked(dist, m), 0);
    if ((cerr = cudaEventRecord(hs.gen_done[h], stream)) != cudaSuccess) break;
    if ((cerr = cudaStreamWaitEvent(hs.copy_stream, hs.gen_done[h], 0)) != cudaSuccess) break;
    if ((cerr = cudaMemcpyAsync(host + (size_t)done * (size_t)es, half, (size_t)m * (size_t)es,
                                cudaMemcpyDeviceToHost, hs.copy_stream)) != cudaSuccess)
      break;
    if ((cerr = cudaEventRecord(hs.copy_done[h], hs.copy_stream)) != cudaSuccess) break;
    done += m;
    ++idx;
  }
  const cudaError_t serr = cudaStreamSynchronize(hs.copy_stream);
  if (st != GRNG_OK) return st;
  if (cerr == cudaSuccess) cerr = serr;
  if (cerr != cudaSuccess) {
    set_error("generate_host: %s", cudaGetErrorString(cerr));
    cudaGetLastError();
    return GRNG_ERR_CUDA;
  }
  *engine = local;
  return GRNG_OK;
}

}  // extern "C"
