/*
 * grng.h - C ABI of a GB300 (sm_103a) bulk random number library.
 *
 * The interface follows the engine / distribution / generate shape of the
 * oneMKL RNG domain that the paper extends (Sec. 4.1: engine classes with
 * `generate` templates parameterised by a distribution object that carries
 * its own parameters and a custom range), and the native generator flow of
 * Sec. 4.2 (create a generator, set seed and offset, generate into device
 * memory, destroy).  The paper's generate(distr, n, r) call (Sec. 4.3,
 * Listing 1) followed by a separate range-transform kernel (Sec. 4.3,
 * Listing 2) becomes one call and one kernel here: the transform is fused
 * into the generator.
 *
 * Conventions for every function:
 *   - Return value: a grng_status; GRNG_OK (0) on success.  No function
 *     aborts, prints or throws.  On any error the engine is left unchanged.
 *   - Device pointers must belong to the CUDA device that is current on the
 *     calling thread; streams (grng_stream_t, ABI-compatible with
 *     cudaStream_t; NULL = the legacy default stream) likewise.
 *   - Generation calls are asynchronous with respect to the host: they only
 *     enqueue work on `stream`; the output is valid once the stream reaches
 *     that point.  Ordering with other work is stream order.
 *   - The library owns engines (small host structs, no device memory);
 *     callers own every buffer and stream they pass in.
 *   - An engine must not be used by two threads at the same time.  Distinct
 *     engines may be used concurrently.
 *
 * Word streams.  An engine is a stream of 32-bit words w_0, w_1, ... with a
 * 128-bit word offset.  Philox4x32-10 (Salmon et al., SC'11): key =
 * (seed mod 2^32, seed >> 32); word g is lane (g mod 4) of the block whose
 * 128-bit counter is floor(g / 4).  MRG32k3a (L'Ecuyer 1999): seeded state
 * x1 = (1, 1, seed mod m1), x2 = (1, 1, 1); word n is (x1_n - x2_n) mod m1.
 * The paper names both engines (Sec. 4.1) but defines neither.  Offsets
 * are taken mod 2^128: for Philox word 2^128 + g is word g; an MRG32k3a fill
 * whose words cross 2^128 within one call continues its recursion, and the
 * engine's next offset is reduced mod 2^128.
 *
 * Words per output (the consumption rule; the paper does not fix one):
 *   bits U32: 1 | uniform F32: 1 | uniform F64: 2 (the earlier word is the
 *   high half) | gaussian / lognormal F32: 1, F64: 2, consumed in
 *   Box-Muller pairs: an odd n still consumes its last pair whole |
 *   ICDF gaussian / lognormal F32: 1, F64: 2 (no pairing).
 */
#ifndef GRNG_H
#define GRNG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GRNG_API __attribute__((visibility("default")))
#else
#define GRNG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum grng_status {
  GRNG_OK = 0,
  GRNG_ERR_INVALID_ARG = 1, /* null pointer, bad enum, bad parameter, misaligned pointer */
  GRNG_ERR_UNSUPPORTED = 2, /* valid request the library cannot serve (size limits) */
  GRNG_ERR_OOM = 3,         /* host allocation failed */
  GRNG_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  GRNG_ERR_TIMEOUT = 5,     /* reserved for bounded device waits */
  GRNG_ERR_BUDGET = 6       /* reserved for admission budgets */
} grng_status;

typedef enum grng_engine_kind {
  GRNG_PHILOX4X32X10 = 0,
  GRNG_MRG32K3A = 1
} grng_engine_kind;

typedef enum grng_dist_kind {
  GRNG_BITS = 0,      /* raw 32-bit words; dtype must be GRNG_U32 */
  GRNG_UNIFORM = 1,   /* [p0, p1) = [a, b) */
  GRNG_GAUSSIAN = 2,  /* Box-Muller; p0 = mean, p1 = stddev > 0 */
  GRNG_LOGNORMAL = 3, /* exp(m + s z), z Box-Muller; p0 = m, p1 = s > 0 */
  GRNG_GAUSSIAN_ICDF = 4,  /* inverse-CDF method; p0 = mean, p1 = stddev > 0 */
  GRNG_LOGNORMAL_ICDF = 5  /* exp(m + s z), z by the inverse-CDF method */
} grng_dist_kind;

typedef enum grng_dtype { GRNG_U32 = 0, GRNG_F32 = 1, GRNG_F64 = 2 } grng_dtype;

/*
 * A distribution with its parameters (Sec. 4.1: distribution objects carry
 * mean / standard deviation or a custom range).  For F32 outputs the
 * parameters are first rounded to float.
 *   uniform:  u = (w >> 8) 2^-24 (F32) or ((w_a << 32 | w_b) >> 11) 2^-53
 *             (F64); r = a + (b - a) u with round-to-nearest multiply and add
 *             and no fused multiply-add (the range transform of Sec. 4.3,
 *             Listing 2); r >= b is replaced by the largest value below b.
 *             Requires finite a < b with b - a finite in the output type.
 *   gaussian: pair k -> u1 in (0, 1] from its first unit, u2 in [0, 1) from its
 *             second; z0 = rho cos(2 pi u2), z1 = rho sin(2 pi u2),
 *             rho = sqrt(-2 ln u1); output mean + stddev z.
 *   lognormal: exp(m + s z) with z as for gaussian.
 *   gaussian / lognormal ICDF (oneMKL's icdf method, which cuRAND offers
 *             only for quasi-random generators, Sec. 4.1): one uniform per
 *             output, u = (k + 1/2) 2^-23 with k = w >> 9 (F32) or
 *             u = (x + 1/2) 2^-52 with x = ((w_a << 32 | w_b) >> 12) (F64),
 *             z = Phi^-1(u) (F32: x P(-log2(1 - x^2)) with x = 2u - 1, two
 *             polynomial branches as in Giles's erfinv; F64: a fixed-point
 *             piecewise polynomial in sqrt(-2 ln min(u, 1 - u))).
 * Uniform and bits outputs are bit-exact functions of the words; gaussian and
 * lognormal outputs are within 2e-6 max(1, |x|) (F32) or 1e-14 max(1, |x|)
 * (F64) of the exact value (F64 lognormal: for |s z| up to about 10; beyond
 * that the error of z grows with s z, as for any double z).
 */
typedef struct grng_distribution {
  int32_t kind;  /* grng_dist_kind */
  int32_t dtype; /* grng_dtype */
  double p0;
  double p1;
} grng_distribution;

/* Serialisable engine state (checkpoint / resume). */
typedef struct grng_engine_state {
  int32_t kind;        /* grng_engine_kind */
  uint32_t reserved;   /* number of MRG32k3a seed words in words[] (0: seeded by seed) */
  uint64_t seed;       /* the seed, or the Philox key of a word-seeded Philox engine */
  uint64_t offset_lo;  /* 128-bit word offset = offset_lo + 2^64 offset_hi */
  uint64_t offset_hi;
  uint32_t words[6];   /* MRG32k3a seed words (see grng_engine_create_words) */
} grng_engine_state;

typedef struct grng_engine* grng_engine_t;
typedef struct CUstream_st* grng_stream_t; /* same type as cudaStream_t */

/* Human-readable name of a status code (static storage; never NULL).  The
 * paper's generate wraps each native call in a status check (Sec. 4.3,
 * Listing 1: CURAND_CALL and CUDA_CALL take a status variable); here every
 * entry point returns that status instead. */
GRNG_API const char* grng_status_string(grng_status status);

/* Detail of the last error raised on the calling thread (static per-thread
 * storage, overwritten by the next failing call; "" if none).  A reading,
 * not in the paper: the text behind a failing status of Sec. 4.3's calls. */
GRNG_API const char* grng_last_error(void);

/*
 * Creates an engine of `kind` seeded with `seed`, positioned at word offset
 * `offset` (Sec. 4.2: create the generator, then set seed and offset).
 * *out receives the handle; release it with grng_engine_destroy.
 * Errors: INVALID_ARG (out NULL, bad kind), OOM.
 */
GRNG_API grng_status grng_engine_create(grng_engine_t* out, int32_t kind, uint64_t seed, uint64_t offset);

/*
 * Creates an engine from a seed initializer list of `count` (1..6) 32-bit
 * words (oneMKL engines accept such lists; cuRAND's do not, Sec. 4.1):
 *   Philox4x32-10: words 0, 1 = key (k0, k1); words 2..5 = the starting
 *     128-bit block counter (c0..c3; missing words 0), i.e. word offset
 *     4 * counter (mod 2^128) + offset.  {lo, hi} equals seed lo + 2^32 hi.
 *   MRG32k3a: words 0..2 = x1_{-1}, x1_{-2}, x1_{-3} (mod m1) and words 3..5 =
 *     x2_{-1}, x2_{-2}, x2_{-3} (mod m2); missing words are 1, so {w} equals
 *     the single seed w.  A component state of all zeros is INVALID_ARG.
 */
GRNG_API grng_status grng_engine_create_words(grng_engine_t* out, int32_t kind,
                                              const uint32_t* words, int32_t count,
                                              uint64_t offset);

/* Creates an engine from a saved state (checkpoint / resume). */
GRNG_API grng_status grng_engine_restore(grng_engine_t* out, const grng_engine_state* state);

/* Copies an engine (same kind, seed and offset; independent afterwards).
 * oneMKL engines are copy-constructible (Sec. 4.1), cuRAND's are not. */
GRNG_API grng_status grng_engine_copy(grng_engine_t* out, grng_engine_t src);

/* Advances the engine by n = n_lo + 2^64 n_hi words (mod 2^128).  The next
 * generate call starts at the new offset.  Sec. 4.2 sets the offset as a
 * generator option at creation; this sets it later, by the same rule (a
 * reading: the unit of the offset is a 32-bit word).
 * Errors: INVALID_ARG (NULL engine). */
GRNG_API grng_status grng_engine_skip_ahead(grng_engine_t engine, uint64_t n_lo, uint64_t n_hi);

/* Writes the engine's kind, seed, seed words and 128-bit word offset to *out
 * (checkpoint / resume; grng_engine_restore reads it back).  The state is
 * what Sec. 4.2's generator options set (seed, offset); saving it is a
 * reading, not in the paper.  Errors: INVALID_ARG (NULL engine or out). */
GRNG_API grng_status grng_engine_get_state(grng_engine_t engine, grng_engine_state* out);

/* Releases an engine (Sec. 4.2, step 5: the generator's destructor).  NULL
 * is accepted and ignored. */
GRNG_API grng_status grng_engine_destroy(grng_engine_t engine);

/* Number of words that n outputs of `dist` consume (written to *words_out):
 * the consumption rule above.  A reading, not in the paper, which fixes no
 * rule; shard boundaries and continuation offsets are computed from it.
 * Errors: INVALID_ARG (NULL dist or words_out, bad kind / dtype pairing,
 * bad parameters, n < 0), UNSUPPORTED (n > 2^40). */
GRNG_API grng_status grng_words_for(const grng_distribution* dist, int64_t n, uint64_t* words_out);

/*
 * Fills dev_ptr[0 .. n) with n outputs of `dist` drawn from the engine's
 * words starting at its current offset, then advances the engine's offset by
 * grng_words_for(dist, n) words (at enqueue time, like a oneMKL engine that
 * continues its sequence).  One kernel launch on `stream`; no allocation,
 * no synchronisation.
 *   dev_ptr: device memory of n elements of the dtype (uint32 / float /
 *            double), aligned to the element size; any other alignment and
 *            any word offset are accepted.  May be NULL only when n == 0.
 *   n == 0:  no-op, returns GRNG_OK, engine unchanged.
 * Errors: INVALID_ARG (NULL engine/dist, bad kind/dtype pairing, bad
 * parameters, n < 0, misaligned or NULL dev_ptr), UNSUPPORTED (n > 2^40),
 * CUDA (launch failed; engine unchanged).
 */
GRNG_API grng_status grng_generate(const grng_distribution* dist, grng_engine_t engine, int64_t n,
                          void* dev_ptr, grng_stream_t stream);

/*
 * Substream fill in one launch: for s in [0, num_streams), fills
 * dev_ptr[s * n_per_stream .. (s + 1) * n_per_stream) with n_per_stream
 * outputs starting at word offset  offset + s * stride  of the engine, where
 * offset is the engine's current offset and stride = stride_lo + 2^64
 * stride_hi words (e.g. 2^76 for MRG32k3a substreams, 2^40 for Philox).
 * The engine's offset is not changed.  Same argument rules as grng_generate;
 * UNSUPPORTED if num_streams * n_per_stream > 2^40 or num_streams > 2^31.
 */
GRNG_API grng_status grng_generate_substreams(const grng_distribution* dist, grng_engine_t engine,
                                     int64_t n_per_stream, int64_t num_streams,
                                     uint64_t stride_lo, uint64_t stride_hi, void* dev_ptr,
                                     grng_stream_t stream);

/*
 * Applies `dist` to caller-supplied words: dev_out[0 .. n) receives the n
 * outputs that grng_generate would produce from the word sequence
 * dev_words[0 .. grng_words_for(dist, n)) (the transform of Sec. 4.3,
 * Listing 2 and of the distribution objects of Sec. 4.1, without an engine).
 * For bit sources other than the two engines, and for checking the
 * transforms on chosen inputs.  dev_words: device memory, 4-byte aligned,
 * owned by the caller.  Same errors as grng_generate (no engine involved).
 */
GRNG_API grng_status grng_transform_words(const grng_distribution* dist, const uint32_t* dev_words,
                                          int64_t n, void* dev_out, grng_stream_t stream);

/*
 * The RNG-burner flow of Sec. 5.1 / Sec. 7 (generate, then copy the output
 * to the host): fills host_ptr[0 .. n) like grng_generate, staging through
 * the caller's device buffer dev_work of work_bytes bytes (at least 2 MiB,
 * 256-byte aligned), chunk by chunk, copying each chunk device-to-host on
 * `stream` while the next chunk is generated.  host_ptr should be pinned
 * (cudaHostAlloc / cudaHostRegister) for full speed; pageable memory works.
 * Returns after the copies have completed (synchronises `stream`).  The
 * engine advances as one grng_generate(dist, n) would, and the values equal
 * those of that call.
 */
GRNG_API grng_status grng_generate_host(const grng_distribution* dist, grng_engine_t engine, int64_t n,
                               void* host_ptr, void* dev_work, size_t work_bytes,
                               grng_stream_t stream);

/* ---------------------------------------------------------- fill geometry
 * Launch geometry of grng_generate / grng_generate_substreams, one integer
 * per (engine kind, distribution variant, size bucket = bit length of the
 * element count): Philox4x32-10, the CTAs per SM of its grid-stride kernels
 * (1..16: a cap on the resident CTAs; 17..64: value - 16 waves of resident
 * CTAs); MRG32k3a, the threads per SM of the chunk plan in units of 256 (sets
 * the chunk length); 0 = the built-in choice (Philox: 8 waves of resident
 * CTAs; MRG32k3a: 2048 threads per SM).  Tuning is
 * what the paper expects of kernels written for the hardware (Sec. 8; Sec. 7
 * shows the launch configuration mattering).  Outputs never depend on the
 * geometry.  The table starts from the file named by the environment
 * variable GRNG_TUNE_CACHE, if it exists, when first read.  The table is
 * process-wide; the calls below may race with fills on other threads only
 * in which geometry those fills use.
 */

/* Times a fill of n outputs of `dist` into dev_buf (caller-owned device
 * memory of n elements, aligned to the element size) at each candidate
 * geometry (Philox: 0, 1, 2, 4, 17, 18, 20, 32, 48, 64; MRG32k3a: 0, 1, 2, 4,
 * 6, 12, 16),
 * with a private engine (no caller engine moves), and keeps the fastest for
 * n's bucket (a candidate must beat the earlier best by 1 %, so ties keep the
 * built-in choice); *best_geometry, *best_ms and *builtin_ms (the built-in
 * choice's time; each may be NULL) receive the result.  Synchronises
 * `stream`.  Errors: INVALID_ARG (bad kind, dist, n < 1, NULL dev_buf), CUDA. */
GRNG_API grng_status grng_fill_autotune(int32_t engine_kind, const grng_distribution* dist,
                                        int64_t n, void* dev_buf, grng_stream_t stream,
                                        int32_t* best_geometry, float* best_ms,
                                        float* builtin_ms);

/* Sets / reads the geometry of n's bucket (0..64; 0 = built-in). */
GRNG_API grng_status grng_fill_set_geometry(int32_t engine_kind, const grng_distribution* dist,
                                            int64_t n, int32_t geometry);
GRNG_API grng_status grng_fill_get_geometry(int32_t engine_kind, const grng_distribution* dist,
                                            int64_t n, int32_t* geometry);

/* Writes the table's non-default entries to `path` ("grng-tune 1", then one
 * "engine variant bucket geometry" line per entry), reads such a file into
 * the table, or resets every entry to 0. */
GRNG_API grng_status grng_tune_save(const char* path);
GRNG_API grng_status grng_tune_load(const char* path);
GRNG_API grng_status grng_tune_reset(void);

/* ------------------------------------------------------------------ batches
 * Many independent requests in one persistent launch: the event batching the
 * paper names as future work for FastCaloSim (Sec. 7), where per-call
 * overheads dominate small batches (Sec. 7, Figs. 2-4).  Requests of one
 * engine follow each other in its sequence in table order, exactly as the
 * same grng_generate calls would.  Engine state for the batch lives on the
 * device: every launch fills every request from its current device offset
 * and then advances each engine by the words of all its requests, so a
 * replayed launch (for example from a CUDA graph that captured
 * grng_batch_launch) continues every sequence without host work.
 * Philox4x32-10 engines only.
 */
typedef struct grng_request {
  grng_engine_t engine;   /* Philox engine; read at grng_batch_create */
  grng_distribution dist;
  int64_t n;              /* outputs */
  void* out;              /* device memory, aligned to the element size */
} grng_request;

typedef struct grng_batch* grng_batch_t;

/* Device workspace a batch of `count` requests needs with `ipt` 16-byte
 * groups per thread per tile (1..64); written to *bytes. */
GRNG_API grng_status grng_batch_workspace_bytes(const grng_request* reqs, int32_t count,
                                                int32_t ipt, size_t* bytes);

/* Plans the batch and uploads its tables (request records, per-request
 * offsets, tile map) into dev_workspace (caller-owned, 256-byte aligned, at
 * least grng_batch_workspace_bytes).  Synchronises `stream` once.  The
 * engines are read, not advanced (see grng_batch_commit).  The workspace
 * must stay alive and untouched while the batch exists. */
GRNG_API grng_status grng_batch_create(grng_batch_t* out, const grng_request* reqs, int32_t count,
                                       int32_t ipt, void* dev_workspace, size_t workspace_bytes,
                                       grng_stream_t stream);

/* Enqueues the fill kernel and the offset-advance kernel on `stream`: no host
 * synchronisation, no allocation; may be captured into a CUDA graph. */
GRNG_API grng_status grng_batch_launch(grng_batch_t batch, grng_stream_t stream);

/* The autotuner of the batched fill (Sec. 8 names tuning as the cost of
 * portable native kernels; Sec. 7 shows small batches dominated by per-call
 * overheads).  Times the fill over the launch geometries ipt (16-byte groups
 * per thread per tile: 1, 2, 4, 8, 16, 32) x CTAs per SM (1, 2, 4, 6, 8, 12,
 * 16), without advancing the offsets (the outputs are rewritten
 * identically), and keeps the fastest.  Only the ipt values whose tile map
 * fits the workspace given to grng_batch_create are tried: a workspace of
 * grng_batch_workspace_bytes(..., ipt = 1, ...) admits every one.  The
 * output never depends on the geometry.  *best_ipt, *best_ctas and *best_ms
 * (each may be NULL) receive the choice.  Synchronises `stream`.  A CUDA
 * graph captured before a change of ipt must be captured again. */
GRNG_API grng_status grng_batch_autotune(grng_batch_t batch, grng_stream_t stream,
                                         int32_t* best_ipt, int32_t* best_ctas, float* best_ms);

/* Sets the fill's geometry (ipt 1..64, CTAs per SM 1..32), e.g. from a
 * saved tuning; re-plans the tile map in the workspace when ipt changes
 * (synchronising `stream`).  INVALID_ARG if that map does not fit. */
GRNG_API grng_status grng_batch_set_config(grng_batch_t batch, int32_t ipt, int32_t ctas_per_sm,
                                           grng_stream_t stream);

/* Moves each engine of the batch to its device-resident offset (after the
 * launches so far).  Synchronises `stream`. */
GRNG_API grng_status grng_batch_commit(grng_batch_t batch, grng_stream_t stream);

/* Releases the plan (not the workspace).  NULL is ignored. */
GRNG_API grng_status grng_batch_destroy(grng_batch_t batch);

/* ------------------------------------------------------------------ serving
 * A continuous-batching server for FastCaloSim-shaped demand (Sec. 5.2: each
 * event needs three uniforms per calorimeter hit, thousands of hits; Sec. 7
 * names event batching as the way to use the GPU).  Requests arrive at any
 * time; a scheduler thread admits them in arrival order while their outputs
 * fit a device-memory budget, packs the admitted ones into one batched
 * launch per free stream slot, and stamps each request complete from a host
 * callback.  Batches on different streams overlap on the device.
 */
#define GRNG_SERVE_AUTO_RELEASE 1 /* free outputs at completion (throughput runs) */

typedef struct grng_serve_part {
  grng_distribution dist;
  int64_t n;
} grng_serve_part;

/* One request: up to four parts drawn in turn from one Philox4x32-10 engine
 * (key = seed, first part at word offset offset_lo + 2^64 offset_hi, each
 * next part after the words of the previous ones).  The output buffer holds
 * the parts one after another, each aligned to its element size. */
typedef struct grng_serve_request {
  uint64_t seed;
  uint64_t offset_lo, offset_hi;
  int32_t num_parts; /* 1..4 */
  int32_t reserved;
  grng_serve_part parts[4];
} grng_serve_request;

typedef struct grng_serve_stats {
  int64_t submitted, completed, rejected, samples, batches;
  double wall_s;             /* first arrival to last completion */
  double latency_p50_us, latency_p90_us, latency_p99_us, latency_max_us, latency_mean_us;
  double peak_pool_bytes;    /* high-water mark of admitted output bytes */
  double mean_batch_requests;
  double admit_wait_p50_us, admit_wait_p99_us, admit_wait_max_us; /* arrival to admission */
} grng_serve_stats;

typedef struct grng_server* grng_server_t;

/* Creates a server over the caller's device pool (256-byte aligned; batch
 * tables for each stream slot take ~1.7 MB at its start, the rest is the
 * output budget).  num_streams: 1..8 stream slots.  flags:
 * GRNG_SERVE_AUTO_RELEASE or 0.  Starts the scheduler thread.  The pool must
 * outlive the server. */
GRNG_API grng_status grng_server_create(grng_server_t* out, void* dev_pool, size_t pool_bytes,
                                        int32_t num_streams, int32_t flags);

/* Queues a request and returns at once with its ticket.  BUDGET if the
 * request alone can never fit the budget; INVALID_ARG for a bad request. */
GRNG_API grng_status grng_server_submit(grng_server_t server, const grng_serve_request* req,
                                        uint64_t* ticket);

/* Waits up to timeout_us for a request; on completion *dev_out / *bytes
 * (either may be NULL) locate its output in the pool.  TIMEOUT if not done. */
GRNG_API grng_status grng_server_wait(grng_server_t server, uint64_t ticket, int64_t timeout_us,
                                      void** dev_out, size_t* bytes);

/* Returns a completed request's output space to the budget. */
GRNG_API grng_status grng_server_release(grng_server_t server, uint64_t ticket);

/* Waits up to timeout_us until nothing is queued or running. */
GRNG_API grng_status grng_server_drain(grng_server_t server, int64_t timeout_us);

/* Counters, arrival-to-completion latency and arrival-to-admission wait
 * percentiles since creation or the last reset. */
GRNG_API grng_status grng_server_stats(grng_server_t server, grng_serve_stats* out);
GRNG_API grng_status grng_server_reset_stats(grng_server_t server);

/* With GRNG_SERVE_AUTO_RELEASE, keeps each completed output in the budget
 * for delay_us microseconds after its completion before freeing it (a
 * consumer that holds every output that long; 0, the default, frees at
 * completion).  When outputs arrive faster than they are let go, the budget
 * binds and admission waits.  A reading of Sec. 5.2's event-by-event demand,
 * not in the paper.  Errors: INVALID_ARG (NULL server, delay_us < 0). */
GRNG_API grng_status grng_server_set_release_delay(grng_server_t server, int64_t delay_us);

/* Submits reqs[i] at arrival_s[i] * time_scale seconds after the call (a
 * trace replay driven from the calling thread); returns after the last
 * submission.  Requests that can never fit are counted as rejected. */
GRNG_API grng_status grng_server_replay(grng_server_t server, const double* arrival_s,
                                        const grng_serve_request* reqs, int64_t count,
                                        double time_scale);

/* Stops the scheduler (requests not yet launched are abandoned), waits for
 * the running batches and releases the server.  Drain first to finish
 * everything submitted.  NULL is ignored. */
GRNG_API grng_status grng_server_destroy(grng_server_t server);

/*
 * Size of the library's static device staging array used by
 * grng_generate_host_static (64 MiB, held on every GPU that loads the
 * library until the process exits).
 */
#define GRNG_STATIC_STAGE_BYTES (64u << 20)

/*
 * The paper has no counterpart to this function.  It is grng_generate_host
 * for callers that cannot allocate device memory at the point of the call:
 * an application whose own memory pool already owns the whole device, code
 * that must not call cudaMalloc / cudaFree because they can synchronise the
 * device, or a plug-in whose host forbids device allocations after start-up.
 * Instead of a caller-provided device buffer it stages through a fixed
 * array inside the library (GRNG_STATIC_STAGE_BYTES per device), and it
 * allocates nothing, on the device or the host.
 *
 * Fills host_ptr[0 .. n) like grng_generate(dist, engine, n, ...) followed by
 * a device-to-host copy on `stream`, and returns after the copy completed
 * (synchronises `stream`).  The values and the engine's advance equal those
 * of grng_generate.  host_ptr may be pinned or pageable.
 *   n * element size must not exceed GRNG_STATIC_STAGE_BYTES: larger
 *   requests return GRNG_ERR_UNSUPPORTED (split them into several calls; the
 *   engine continues its sequence across calls).
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and keeps it; make that
 *   first call before any stream capture begins.  Do not use this function
 *   on a device after cudaDeviceReset in the same process: the kept address
 *   would be stale.
 *   All calls share the one array.  The library serialises its own calls
 *   and waits for each copy, so calls from one process do not overlap on the
 *   GPU; calls that did overlap would race on the array.  Nothing in it has
 *   to start at zero: every element copied out is written first.
 * Errors: as grng_generate; UNSUPPORTED above the size limit or for a
 * device ordinal of 256 or more; CUDA if the copy fails (the engine is then
 * moved back to where it was).
 */
GRNG_API grng_status grng_generate_host_static(const grng_distribution* dist,
                                               grng_engine_t engine, int64_t n,
                                               void* host_ptr, grng_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GRNG_H */
