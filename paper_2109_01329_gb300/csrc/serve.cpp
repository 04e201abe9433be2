// Continuous-batching server for generation requests (grng_server_*).
//
// FastCaloSim (Sec. 5.2) asks for random numbers event by event: three
// uniforms per calorimeter hit and thousands of hits per event, with event
// batching named as the way to use the GPU better (Sec. 7).  The server takes
// such requests as they arrive and keeps the GPU busy with them:
//   * submit() queues a request (up to four distribution parts drawn in turn
//     from one Philox4x32-10 engine given by seed and offset) and returns at
//     once;
//   * a scheduler thread admits queued requests in arrival order while their
//     outputs fit in the device-memory budget (a first-fit allocator over the
//     caller's pool), packs every admitted request into one batch and launches
//     it on the next free stream slot (table upload from pinned memory, the
//     batched fill kernel of batch.cu, a host callback), so batches on
//     different streams overlap on the device while new requests keep
//     arriving;
//   * the host callback stamps each request complete (latency = completion -
//     arrival) and frees its slot; outputs stay in the pool until released
//     (or, with GRNG_SERVE_AUTO_RELEASE, at completion plus the release
//     delay: a consumer that keeps each output that long, which makes the
//     budget bind when outputs arrive faster than they are let go).
// No call allocates device memory: the pool and every table live in the
// caller's buffer; pinned staging for the tables is allocated at creation.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "grng.h"
#include "grng_internal.h"

namespace grng {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxParts = 4096;      // parts per batch
constexpr int64_t kMaxTiles = 1 << 18;  // tiles per batch
constexpr int kIpt = 4;              // 16-byte groups per thread per tile
constexpr int kMaxSlots = 8;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, size) in 256-byte granules, coalescing on free.
class PoolAlloc {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes ? bytes : 1, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, noff = it->first + bytes;
      free_.erase(it);
      if (rest) free_[noff] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes ? bytes : 1, 256);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Req {
  grng_serve_request spec;
  size_t bytes = 0;
  size_t part_off[4] = {0, 0, 0, 0};  // byte offset of each part in the output
  int64_t samples = 0;
  int64_t tiles = 0;
  size_t off = 0;                     // pool offset of the output
  int state = 0;                      // 0 queued, 1 launched, 2 done
  Clock::time_point t_arrival, t_admit, t_done;
};

struct Slot {
  cudaStream_t stream = nullptr;
  BatchReq* h_reqs = nullptr;
  uint64_t* h_offs = nullptr;
  int32_t* h_tiles = nullptr;
  BatchReq* d_reqs = nullptr;
  uint64_t* d_offs = nullptr;
  int32_t* d_tiles = nullptr;
  std::vector<uint64_t> tickets;
  bool busy = false;
  struct grng_server* server = nullptr;
};

}  // namespace
}  // namespace grng

using namespace grng;

struct grng_server {
  char* out_base = nullptr;  // start of the output region of the pool
  size_t out_bytes = 0;
  int32_t flags = 0;
  int64_t grid = 1;
  std::mutex mu;
  std::condition_variable cv;       // scheduler: work or space available
  std::condition_variable cv_done;  // waiters: completions
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  PoolAlloc alloc;
  Slot slots[kMaxSlots];
  int32_t num_slots = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread sched;
  cudaError_t async_error = cudaSuccess;
  // automatic releases waiting for their time: deadline -> (offset, bytes)
  int64_t release_delay_us = 0;
  std::multimap<Clock::time_point, std::pair<size_t, size_t>> deferred;
  // statistics
  std::vector<double> lat_us;
  std::vector<double> wait_us;  // arrival to admission
  int64_t submitted = 0, completed = 0, rejected = 0, samples = 0, batches = 0,
          batch_reqs = 0;
  size_t peak_used = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace {

void CUDART_CB on_batch_done(void* arg) {
  Slot* slot = static_cast<Slot*>(arg);
  grng_server* S = slot->server;
  {
    std::lock_guard<std::mutex> g(S->mu);
    const Clock::time_point now = Clock::now();
    for (uint64_t t : slot->tickets) {
      auto it = S->reqs.find(t);
      if (it == S->reqs.end()) continue;
      Req& r = it->second;
      r.state = 2;
      r.t_done = now;
      S->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_arrival).count());
      S->completed += 1;
      S->samples += r.samples;
      S->t_last = now;
      if (S->flags & GRNG_SERVE_AUTO_RELEASE) {
        if (S->release_delay_us > 0)
          S->deferred.emplace(now + std::chrono::microseconds(S->release_delay_us),
                              std::make_pair(r.off, r.bytes));
        else
          S->alloc.release(r.off, r.bytes);
        S->reqs.erase(it);
      }
    }
    slot->tickets.clear();
    slot->busy = false;
  }
  S->cv.notify_all();
  S->cv_done.notify_all();
}

// Frees the automatic releases whose time has come (caller holds S->mu).
void release_due(grng_server* S) {
  const Clock::time_point now = Clock::now();
  while (!S->deferred.empty() && S->deferred.begin()->first <= now) {
    S->alloc.release(S->deferred.begin()->second.first, S->deferred.begin()->second.second);
    S->deferred.erase(S->deferred.begin());
  }
}

// Waits for a submission, a completion or the next automatic release.
void wait_for_work(grng_server* S, std::unique_lock<std::mutex>& lk) {
  if (S->deferred.empty())
    S->cv.wait(lk);
  else
    S->cv.wait_until(lk, S->deferred.begin()->first);
}

void scheduler(grng_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  std::vector<PartDesc> parts;
  parts.reserve(kMaxParts);
  for (;;) {
    release_due(S);
    Slot* slot = nullptr;
    for (int i = 0; i < S->num_slots; ++i)
      if (!S->slots[i].busy) {
        slot = &S->slots[i];
        break;
      }
    if (S->stop) break;  // requests not yet launched are abandoned
    if (slot == nullptr || S->queue.empty()) {
      wait_for_work(S, lk);
      continue;
    }
    // admit in arrival order while the outputs fit the budget
    std::vector<uint64_t> batch;
    int nparts = 0;
    int64_t ntiles = 0;
    const Clock::time_point t_admit = Clock::now();
    while (!S->queue.empty()) {
      Req& r = S->reqs[S->queue.front()];
      if (nparts + r.spec.num_parts > kMaxParts) break;
      if (ntiles + r.tiles > kMaxTiles) break;
      size_t off = 0;
      if (!S->alloc.alloc(r.bytes, &off)) break;
      r.off = off;
      r.state = 1;
      r.t_admit = t_admit;
      S->wait_us.push_back(
          std::chrono::duration<double, std::micro>(t_admit - r.t_arrival).count());
      batch.push_back(S->queue.front());
      S->queue.pop_front();
      nparts += r.spec.num_parts;
      ntiles += r.tiles;
    }
    if (batch.empty()) {  // the oldest request waits for space
      wait_for_work(S, lk);
      continue;
    }
    S->peak_used = std::max(S->peak_used, S->alloc.used());
    slot->busy = true;
    slot->tickets = batch;
    S->batches += 1;
    S->batch_reqs += (int64_t)batch.size();
    parts.clear();
    for (uint64_t t : batch) {
      const Req& r = S->reqs[t];
      uint64_t lo = r.spec.offset_lo, hi = r.spec.offset_hi;
      for (int k = 0; k < r.spec.num_parts; ++k) {
        const grng_serve_part& sp = r.spec.parts[k];
        PartDesc d;
        std::memset(&d, 0, sizeof(d));
        d.key0 = (uint32_t)r.spec.seed;
        d.key1 = (uint32_t)(r.spec.seed >> 32);
        d.off_lo = lo;
        d.off_hi = hi;
        fill_transform_params(&sp.dist, &d.t, &d.variant);
        d.es = sp.dist.dtype == GRNG_F64 ? 8 : 4;
        d.n = sp.n;
        d.out = (uint64_t)(uintptr_t)(S->out_base + r.off + r.part_off[k]);
        parts.push_back(d);
        uint64_t w = 0;
        grng_words_for(&sp.dist, sp.n, &w);
        const uint64_t nlo = lo + w;
        hi += (nlo < lo) ? 1u : 0u;
        lo = nlo;
      }
    }
    lk.unlock();
    // tables -> pinned staging -> device; fill; completion callback
    const int64_t tiles = plan_parts(parts.data(), (int32_t)parts.size(), kIpt, slot->h_reqs,
                                     slot->h_offs, slot->h_tiles, kMaxTiles);
    cudaError_t err = cudaMemcpyAsync(slot->d_reqs, slot->h_reqs, sizeof(BatchReq) * parts.size(),
                                      cudaMemcpyHostToDevice, slot->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(slot->d_offs, slot->h_offs, 16u * parts.size(),
                            cudaMemcpyHostToDevice, slot->stream);
    if (err == cudaSuccess && tiles > 0)
      err = cudaMemcpyAsync(slot->d_tiles, slot->h_tiles, 4u * (size_t)tiles,
                            cudaMemcpyHostToDevice, slot->stream);
    if (err == cudaSuccess &&
        enqueue_fill(slot->d_reqs, slot->d_offs, slot->d_tiles, tiles, kIpt, S->grid,
                     slot->stream) != GRNG_OK)
      err = cudaErrorLaunchFailure;
    if (err == cudaSuccess) err = cudaLaunchHostFunc(slot->stream, on_batch_done, slot);
    lk.lock();
    if (err != cudaSuccess) {
      // record the failure; the batch's requests complete as failed
      S->async_error = err;
      cudaGetLastError();
      for (uint64_t t : slot->tickets) {
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) continue;
        it->second.state = 2;
        it->second.t_done = Clock::now();
        if (S->flags & GRNG_SERVE_AUTO_RELEASE) {
          S->alloc.release(it->second.off, it->second.bytes);
          S->reqs.erase(it);
        }
      }
      slot->tickets.clear();
      slot->busy = false;
      S->cv_done.notify_all();
    }
  }
}

grng_status check_request(const grng_serve_request* q, Req* r) {
  if (q == nullptr || q->num_parts < 1 || q->num_parts > 4) {
    set_error("a request has 1 to 4 parts");
    return GRNG_ERR_INVALID_ARG;
  }
  size_t pos = 0;
  const int64_t tile_groups = 256 * kIpt;
  for (int k = 0; k < q->num_parts; ++k) {
    const grng_serve_part& p = q->parts[k];
    uint64_t w = 0;
    const grng_status st = grng_words_for(&p.dist, p.n, &w);  // checks dist and n
    if (st != GRNG_OK) return st;
    const size_t es = p.dist.dtype == GRNG_F64 ? 8 : 4;
    pos = round_up(pos, es);
    r->part_off[k] = pos;
    const int64_t head = (int64_t)((pos & 15u) / es);  // the output starts 256-byte aligned
    const int64_t groups = p.n == 0 ? 0 : (head + p.n + (int64_t)(16 / es) - 1) / (int64_t)(16 / es);
    r->tiles += (groups + tile_groups - 1) / tile_groups;
    pos += (size_t)p.n * es;
    r->samples += p.n;
  }
  r->bytes = pos;
  r->spec = *q;
  return GRNG_OK;
}

}  // namespace

extern "C" {

grng_status grng_server_create(grng_server_t* out, void* dev_pool, size_t pool_bytes,
                               int32_t num_streams, int32_t flags) {
  if (out == nullptr || dev_pool == nullptr || ((uintptr_t)dev_pool & 255u) != 0 ||
      num_streams < 1 || num_streams > kMaxSlots) {
    set_error("out / pool NULL, pool not 256-byte aligned, or num_streams not in [1, 8]");
    return GRNG_ERR_INVALID_ARG;
  }
  const size_t slot_bytes = round_up(sizeof(BatchReq) * kMaxParts, 256) +
                            round_up(16u * kMaxParts, 256) + round_up(4u * kMaxTiles, 256);
  const size_t tables = slot_bytes * (size_t)num_streams;
  if (pool_bytes < tables + (size_t(1) << 20)) {
    set_error("pool of %zu bytes is below the %zu bytes of tables plus 1 MiB", pool_bytes, tables);
    return GRNG_ERR_INVALID_ARG;
  }
  grng_server* S = new (std::nothrow) grng_server;
  if (S == nullptr) {
    set_error("server allocation failed");
    return GRNG_ERR_OOM;
  }
  char* base = static_cast<char*>(dev_pool);
  S->flags = flags;
  int dev = 0;
  S->grid = (int64_t)current_device_sms(&dev) * 8;
  for (int i = 0; i < num_streams; ++i) {
    Slot& sl = S->slots[i];
    sl.server = S;
    char* d = base + (size_t)i * slot_bytes;
    sl.d_reqs = reinterpret_cast<BatchReq*>(d);
    sl.d_offs = reinterpret_cast<uint64_t*>(d + round_up(sizeof(BatchReq) * kMaxParts, 256));
    sl.d_tiles = reinterpret_cast<int32_t*>(d + round_up(sizeof(BatchReq) * kMaxParts, 256) +
                                            round_up(16u * kMaxParts, 256));
    void* h = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaHostAlloc(&h, slot_bytes, cudaHostAllocDefault);
    if (err != cudaSuccess) {
      set_error("server set-up failed: %s", cudaGetErrorString(err));
      cudaGetLastError();
      for (int j = 0; j <= i; ++j) {
        if (S->slots[j].stream) cudaStreamDestroy(S->slots[j].stream);
        if (S->slots[j].h_reqs) cudaFreeHost(S->slots[j].h_reqs);
      }
      delete S;
      return GRNG_ERR_CUDA;
    }
    char* hc = static_cast<char*>(h);
    sl.h_reqs = reinterpret_cast<BatchReq*>(hc);
    sl.h_offs = reinterpret_cast<uint64_t*>(hc + round_up(sizeof(BatchReq) * kMaxParts, 256));
    sl.h_tiles = reinterpret_cast<int32_t*>(hc + round_up(sizeof(BatchReq) * kMaxParts, 256) +
                                            round_up(16u * kMaxParts, 256));
    S->num_slots = i + 1;
  }
  S->out_base = base + tables;
  S->out_bytes = pool_bytes - tables;
  S->alloc.reset(S->out_bytes);
  S->sched = std::thread(scheduler, S);
  *out = S;
  return GRNG_OK;
}

grng_status grng_server_submit(grng_server_t S, const grng_serve_request* q, uint64_t* ticket) {
  if (S == nullptr || ticket == nullptr) {
    set_error("server or ticket NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  Req r;
  grng_status st = check_request(q, &r);
  if (st != GRNG_OK) return st;
  if (round_up(r.bytes, 256) > S->out_bytes || r.tiles > kMaxTiles ||
      q->num_parts > kMaxParts) {
    std::lock_guard<std::mutex> g(S->mu);
    S->rejected += 1;
    set_error("request of %zu bytes can never fit the %zu-byte budget", r.bytes, S->out_bytes);
    return GRNG_ERR_BUDGET;
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
      set_error("server is stopping");
      return GRNG_ERR_INVALID_ARG;
    }
    r.t_arrival = Clock::now();
    if (!S->have_first) {
      S->have_first = true;
      S->t_first = r.t_arrival;
    }
    const uint64_t t = S->next_ticket++;
    S->reqs.emplace(t, r);
    S->queue.push_back(t);
    S->submitted += 1;
    *ticket = t;
  }
  S->cv.notify_all();
  return GRNG_OK;
}

grng_status grng_server_wait(grng_server_t S, uint64_t ticket, int64_t timeout_us,
                             void** dev_out, size_t* bytes) {
  if (S == nullptr) {
    set_error("server NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("unknown or released ticket");
    return GRNG_ERR_INVALID_ARG;
  }
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  while (true) {
    it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
      set_error("ticket released while waiting");
      return GRNG_ERR_INVALID_ARG;
    }
    if (it->second.state == 2) break;
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = S->reqs.find(ticket);
      if (it != S->reqs.end() && it->second.state == 2) break;
      set_error("request not complete within %lld us", (long long)timeout_us);
      return GRNG_ERR_TIMEOUT;
    }
  }
  if (S->async_error != cudaSuccess) {
    set_error("a batch failed: %s", cudaGetErrorString(S->async_error));
    return GRNG_ERR_CUDA;
  }
  if (dev_out) *dev_out = S->out_base + it->second.off;
  if (bytes) *bytes = it->second.bytes;
  return GRNG_OK;
}

grng_status grng_server_release(grng_server_t S, uint64_t ticket) {
  if (S == nullptr) {
    set_error("server NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second.state != 2) {
      set_error("ticket unknown or not complete");
      return GRNG_ERR_INVALID_ARG;
    }
    S->alloc.release(it->second.off, it->second.bytes);
    S->reqs.erase(it);
  }
  S->cv.notify_all();
  return GRNG_OK;
}

grng_status grng_server_drain(grng_server_t S, int64_t timeout_us) {
  if (S == nullptr) {
    set_error("server NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  auto idle = [S] {
    if (!S->queue.empty()) return false;
    for (int i = 0; i < S->num_slots; ++i)
      if (S->slots[i].busy) return false;
    return true;
  };
  while (!idle()) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !idle()) {
      set_error("server not idle within %lld us", (long long)timeout_us);
      return GRNG_ERR_TIMEOUT;
    }
  }
  if (S->async_error != cudaSuccess) {
    set_error("a batch failed: %s", cudaGetErrorString(S->async_error));
    return GRNG_ERR_CUDA;
  }
  return GRNG_OK;
}

grng_status grng_server_stats(grng_server_t S, grng_serve_stats* out) {
  if (S == nullptr || out == nullptr) {
    set_error("NULL argument");
    return GRNG_ERR_INVALID_ARG;
  }
  std::vector<double> lat;
  std::lock_guard<std::mutex> g(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->samples = S->samples;
  out->batches = S->batches;
  out->mean_batch_requests = S->batches ? (double)S->batch_reqs / (double)S->batches : 0.0;
  out->peak_pool_bytes = (double)S->peak_used;
  out->wall_s = S->have_first && S->completed
                    ? std::chrono::duration<double>(S->t_last - S->t_first).count()
                    : 0.0;
  lat = S->lat_us;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
      size_t i = (size_t)(q / 100.0 * (double)(lat.size() - 1) + 0.5);
      return lat[std::min(i, lat.size() - 1)];
    };
    double sum = 0;
    for (double x : lat) sum += x;
    out->latency_p50_us = pct(50);
    out->latency_p90_us = pct(90);
    out->latency_p99_us = pct(99);
    out->latency_max_us = lat.back();
    out->latency_mean_us = sum / (double)lat.size();
  }
  std::vector<double> w = S->wait_us;
  if (!w.empty()) {
    std::sort(w.begin(), w.end());
    auto pct = [&](double q) {
      size_t i = (size_t)(q / 100.0 * (double)(w.size() - 1) + 0.5);
      return w[std::min(i, w.size() - 1)];
    };
    out->admit_wait_p50_us = pct(50);
    out->admit_wait_p99_us = pct(99);
    out->admit_wait_max_us = w.back();
  }
  return GRNG_OK;
}

grng_status grng_server_set_release_delay(grng_server_t S, int64_t delay_us) {
  if (S == nullptr || delay_us < 0) {
    set_error("server NULL or delay < 0");
    return GRNG_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->release_delay_us = delay_us;
  }
  S->cv.notify_all();
  return GRNG_OK;
}

grng_status grng_server_reset_stats(grng_server_t S) {
  if (S == nullptr) {
    set_error("server NULL");
    return GRNG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> g(S->mu);
  S->lat_us.clear();
  S->wait_us.clear();
  S->submitted = S->completed = S->rejected = S->samples = S->batches = S->batch_reqs = 0;
  S->peak_used = S->alloc.used();
  S->have_first = false;
  return GRNG_OK;
}

grng_status grng_server_replay(grng_server_t S, const double* arrival_s,
                               const grng_serve_request* reqs, int64_t count, double time_scale) {
  if (S == nullptr || (count > 0 && (arrival_s == nullptr || reqs == nullptr)) ||
      !(time_scale > 0)) {
    set_error("bad replay arguments");
    return GRNG_ERR_INVALID_ARG;
  }
  const Clock::time_point t0 = Clock::now();
  for (int64_t i = 0; i < count; ++i) {
    const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                              std::chrono::duration<double>(arrival_s[i] * time_scale));
    std::this_thread::sleep_until(due);
    uint64_t t = 0;
    const grng_status st = grng_server_submit(S, &reqs[i], &t);
    if (st != GRNG_OK && st != GRNG_ERR_BUDGET) return st;
  }
  return GRNG_OK;
}

grng_status grng_server_destroy(grng_server_t S) {
  if (S == nullptr) return GRNG_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->sched.joinable()) S->sched.join();
  for (int i = 0; i < S->num_slots; ++i) {
    cudaStreamSynchronize(S->slots[i].stream);
    cudaStreamDestroy(S->slots[i].stream);
    cudaFreeHost(S->slots[i].h_reqs);
  }
  cudaGetLastError();
  delete S;
  return GRNG_OK;
}

}  // extern "C"
