// pa_server.cu -- continuous-batching solve server.
//
// Requests (one pilot-assignment instance each: L, K, gains, positions,
// seed) arrive at any time through pa_server_submit.  Each pa_server_poll
//   1. harvests the ticks that finished on the GPU (an event per tick, no
//      waiting): their slots advance; requests that reached G generations
//      are queued as completions and their slots stay resident for the next
//      request of the same (L, K) class;
//   2. admits queued requests, in arrival order, into resident slots of
//      their class -- a slot is a resident context (gains, tables, double-
//      buffered population on the GPU); new slots are created while the
//      device memory they need stays within the server's budget (idle slots
//      of other classes are destroyed when the next request needs their
//      memory; at most four are created per poll);
//   3. launches one tick for every active slot that has no tick in flight:
//      the newly admitted ones are seeded (one launch), then each advances
//      by up to `tick` generations in one persistent batched launch per
//      kernel variant (side by side on side streams), and the best members
//      of slots that finish are copied to pinned memory;
//   4. returns queued completions.
// Ticks run on a pool of streams, so a request admitted while another tick
// is on the GPU starts at once on the SMs that tick leaves free instead of
// waiting for it; pa_server_wait blocks until some tick finishes.  A
// request's result is exactly what pa_solve gives for the same instance and
// seed alone: generations run in the same order with the same draws,
// whatever the tick length or the mix.
//
// Liveness: requests are checked at submit (shape, values, a slot of its
// shape within the budget), so every queued request can eventually be
// admitted; an admission that fails anyway completes that request with the
// error and the queue moves on.  No C++ exception crosses the C ABI:
// allocation failures return PA_ENOMEM.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "pa_internal.cuh"

namespace pa {
void set_thread_error(const std::string& msg);
bool config_ok(const pa_config* c, std::string* why);
void f32_geometry(int L, int K, int* NJ, int* RS, int* vec);
}

namespace {
constexpr int kTickPool = 4;     // ticks in flight at most
constexpr int kMaxNewSlots = 4;  // contexts created per poll at most
}  // namespace

struct pa_server {
  pa_config base{};
  int G = 0, tick = 0;
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;  // slot creation; ticks wait for it
  bool own_stream = false;
  struct Slot {
    pa_ctx* ctx = nullptr;  // null: destroyed (entry reusable)
    int L = 0, K = 0;
    size_t bytes = 0;       // device bytes charged to the budget
    int64_t req = -1;
    int gen = 0;
    bool active = false, fresh = false;
    int tick = -1;          // the tick in flight on this slot, or -1
    bool cancelled = false; // withdrawn while its tick was in flight
  };
  std::vector<Slot> slots;
  std::map<std::pair<int, int>, std::vector<int>> free_slots;
  struct Req {
    int64_t id;
    int L, K;
    uint64_t seed;
    std::vector<double> beta;
    std::vector<int32_t> uxy, bxy;
  };
  std::deque<Req> pending;
  struct Done {
    int64_t id;
    pa_status st;
    int L, K;
    std::vector<uint8_t> best;
    double fit;
  };
  std::deque<Done> done;   // completions not yet returned by a poll
  int inject_failures = 0; // testing: admissions still to fail
  // One tick in flight: its stream and completion event, the slots it
  // advances, and its own device/pinned scratch (ticks overlap).
  struct Tick {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr, fork = nullptr;
    bool busy = false;
    bool dirty = false;                // work enqueued by a launch that did not finish
    uint64_t seq = 0;                  // launch order
    std::vector<int> slots, g_now, finish_k;  // per slot: generations (-1: failed), index among finishing (-1)
    std::vector<int> failed;           // slots whose group did not fit (complete with an error)
    std::vector<int64_t> best_off;     // per finishing slot: offset in h_best
    unsigned char* h_stage = nullptr;  // pinned uploads of this tick's admissions
    size_t stage_cap = 0, stage_used = 0;
    void* d_seed_args = nullptr;
    void* h_seed_args = nullptr;
    size_t seed_cap = 0;
    void* d_solve_args = nullptr;
    void* h_solve_args = nullptr;
    size_t solve_cap = 0;
    int* d_counters = nullptr;
    size_t counters_cap = 0;
    uint8_t* h_best = nullptr;
    size_t best_cap = 0;
    double* d_bestfit = nullptr;
    double* h_bestfit = nullptr;
    size_t fit_cap = 0;
    std::vector<cudaStream_t> side;    // variant groups side by side
    std::vector<cudaEvent_t> joined;
  };
  Tick ticks[kTickPool];
  uint64_t tick_seq = 0;
  std::vector<std::tuple<int, int, int, int>> prepared;  // kernel variants already loaded
  std::string err;
  int64_t completed = 0;
};

namespace {

pa_status sfail(pa_server* s, pa_status st, const std::string& m) {
  if (s) s->err = m;
  return st;
}

pa_status scuda(pa_server* s, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PA_OK;
  return sfail(s, e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

// Configuration of a request's slot.
pa_config slot_config(const pa_server* s, int L, int K) {
  pa_config c = s->base;
  c.L = L;
  c.K = K;
  c.tau_p = K;
  c.kmeans_k = K;
  return c;
}

// The batched solve kernel runs this shape for some cluster size (tables in
// shared memory, member records within one CTA's share).
bool shape_runs(const pa_config& c) {
  pa_ctx t;  // geometry only: no device memory behind it
  t.cfg = c;
  if (c.prec == PA_FP32) {
    if (!pa::f32_supported(c.L, c.K, nullptr)) return false;
    pa::f32_geometry(c.L, c.K, &t.t32.NJ, &t.t32.RS, &t.t32.vec);
  }
  unsigned char args[512];
  if (pa::solve_args_bytes() > sizeof args) return false;
  for (int C : {16, 8, 4, 2, 1})
    if (pa::solve_fill_args(&t, C, 0, 1, nullptr, nullptr, nullptr, nullptr, nullptr, args) != 0)
      return true;
  return false;
}

// Device bytes a context of this shape allocates (upper estimate).
size_t slot_bytes(const pa_config& c) {
  const size_t L = c.L, K = c.K, LK = L * K, N = c.N;
  size_t b = 8 * L * LK + 8 * L;                 // beta, bnc
  b += 4 * (LK * (L + 8) + LK + L + 16);         // FP32 tables (generous row stride)
  b += 4 * 2 * LK + 4 * 2 * L + 4 * LK;          // positions, labels
  b += 8 * 2 * c.kmeans_k + 2 * N * LK + 8 * N;  // centroids, populations, fitness
  b += 64 + LK;                                  // scratch, best row
  return b + 8 * 256;                            // allocation granularity slack
}

// Grow a device buffer (dev) and/or a pinned host buffer (host) to `need`
// bytes (geometric growth: pinned allocations are slow).  Only called on a
// tick that is not in flight.
template <typename T>
pa_status grow(pa_server* s, T** dev, T** host, size_t* cap, size_t need) {
  if (need <= *cap) return PA_OK;
  const size_t n = std::max(need, *cap * 2 + 64);
  if (dev) {
    cudaFree(*dev);
    *dev = nullptr;
  }
  if (host) {
    cudaFreeHost(*host);
    *host = nullptr;
  }
  *cap = 0;
  if (dev) {
    pa_status st = scuda(s, cudaMalloc(dev, n), "cudaMalloc server scratch");
    if (st != PA_OK) return st;
  }
  if (host) {
    pa_status st = scuda(s, cudaMallocHost(host, n), "cudaMallocHost server scratch");
    if (st != PA_OK) return st;
  }
  *cap = n;
  return PA_OK;
}

// Make sure tick t has a stream, events and k side streams.
pa_status tick_streams(pa_server* s, pa_server::Tick& t, size_t k) {
  if (!t.st) {
    pa_status st = scuda(s, cudaStreamCreateWithFlags(&t.st, cudaStreamNonBlocking), "stream");
    if (st == PA_OK) st = scuda(s, cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming), "event");
    if (st == PA_OK) st = scuda(s, cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming), "event");
    if (st != PA_OK) return st;
  }
  while (t.side.size() < k) {
    cudaStream_t x = nullptr;
    cudaEvent_t e = nullptr;
    pa_status st = scuda(s, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "stream");
    if (st != PA_OK) return st;
    st = scuda(s, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    if (st != PA_OK) {
      cudaStreamDestroy(x);
      return st;
    }
    t.side.push_back(x);
    t.joined.push_back(e);
  }
  return PA_OK;
}

// Queue a completion (a failed one: no best member, NaN fitness).
void complete(pa_server* s, int64_t id, pa_status st, int L, int K, const uint8_t* best,
              double fit) {
  pa_server::Done d;
  d.id = id;
  d.st = st;
  d.L = L;
  d.K = K;
  d.best.assign((size_t)L * K, 0);
  if (best) std::memcpy(d.best.data(), best, (size_t)L * K);
  d.fit = st == PA_OK ? fit : std::nan("");
  s->done.push_back(std::move(d));
  ++s->completed;
}

// A slot is idle again: back to its class's free list (its context on the
// server stream, so that destroying it never waits for a tick stream).
void release(pa_server* s, int i) {
  pa_server::Slot& sl = s->slots[i];
  sl.active = false;
  sl.fresh = false;
  sl.cancelled = false;
  sl.req = -1;
  sl.tick = -1;
  sl.ctx->stream = s->stream;
  s->free_slots[std::make_pair(sl.L, sl.K)].push_back(i);
}

// Destroy one idle slot and give its memory back to the budget.
void evict(pa_server* s, int i) {
  pa_server::Slot& sl = s->slots[i];
  pa_destroy(sl.ctx);
  sl.ctx = nullptr;
  s->used -= sl.bytes;
  sl.bytes = 0;
}

// Destroy idle slots (other classes than `key` first) until `need` more
// bytes fit the budget; true when they do.
bool make_room(pa_server* s, size_t need, std::pair<int, int> key) {
  for (int pass = 0; pass < 2 && s->used + need > s->budget; ++pass)
    for (auto& kv : s->free_slots) {
      if ((kv.first == key) != (pass == 1)) continue;
      while (!kv.second.empty() && s->used + need > s->budget) {
        evict(s, kv.second.back());
        kv.second.pop_back();
      }
    }
  return s->used + need <= s->budget;
}

void destroy_server(pa_server* s) {
  if (!s) return;
  // drain every tick, then destroy the slot contexts (whose stream may still
  // name a tick stream), then the ticks' streams and buffers
  for (auto& t : s->ticks)
    if (t.st) cudaStreamSynchronize(t.st);
  for (auto& sl : s->slots)
    if (sl.ctx) {
      sl.ctx->stream = s->stream;
      pa_destroy(sl.ctx);
      sl.ctx = nullptr;
    }
  for (auto& t : s->ticks) {
    for (auto x : t.side) cudaStreamDestroy(x);
    for (auto e : t.joined) cudaEventDestroy(e);
    if (t.st) cudaStreamDestroy(t.st);
    if (t.ev) cudaEventDestroy(t.ev);
    if (t.fork) cudaEventDestroy(t.fork);
    cudaFreeHost(t.h_stage);
    cudaFree(t.d_seed_args);
    cudaFreeHost(t.h_seed_args);
    cudaFree(t.d_solve_args);
    cudaFreeHost(t.h_solve_args);
    cudaFree(t.d_counters);
    cudaFreeHost(t.h_best);
    cudaFree(t.d_bestfit);
    cudaFreeHost(t.h_bestfit);
  }
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

// First slot of a kernel variant: load every batched-kernel shape a tick
// may choose for it (both column splits, every cluster size) and cache
// their occupancy now -- loading a kernel on its first launch would stall a
// tick by tens of milliseconds.
void prepare_variant(pa_server* s, const pa_ctx* c) {
  const auto key = std::make_tuple(c->cfg.prec, c->cfg.mode, c->t32.NJ, c->t32.vec);
  if (std::find(s->prepared.begin(), s->prepared.end(), key) != s->prepared.end()) return;
  s->prepared.push_back(key);
  std::vector<unsigned char> args(pa::solve_args_bytes());
  for (bool latency : {true, false})
    for (int C : {16, 8, 4, 2, 1}) {
      const size_t smem = pa::solve_fill_args(c, C, 0, 1, nullptr, nullptr, nullptr, nullptr,
                                              nullptr, args.data(), latency);
      if (smem) (void)pa::solve_batch_max_clusters(c, C, smem, latency);
    }
  (void)cudaGetLastError();
}

// Bytes of pinned staging for one request's upload, 16-byte aligned parts.
size_t stage_bytes(const pa_server::Req& r) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  return al(8 * r.beta.size()) + al(4 * r.uxy.size()) + al(4 * r.bxy.size());
}

// A tick whose event has fired: advance its slots, queue the finished
// requests, release their slots.
void finalize(pa_server* s, pa_server::Tick& t) {
  for (size_t m = 0; m < t.slots.size(); ++m) {
    if (t.g_now[m] < 0) continue;  // its group failed: below
    const int i = t.slots[m];
    pa_server::Slot& sl = s->slots[i];
    sl.tick = -1;
    sl.fresh = false;
    sl.gen += t.g_now[m];
    sl.ctx->cur ^= 1;
    sl.ctx->generation = sl.gen;
    const int k = t.finish_k[m];
    if (sl.cancelled) {
      release(s, i);
    } else if (k >= 0) {
      complete(s, sl.req, PA_OK, sl.L, sl.K, t.h_best + t.best_off[k], t.h_bestfit[k]);
      release(s, i);
    }
  }
  for (int i : t.failed) {  // released without a result
    pa_server::Slot& sl = s->slots[i];
    if (!sl.cancelled) complete(s, sl.req, PA_EUNSUPPORTED, sl.L, sl.K, nullptr, 0.0);
    release(s, i);
  }
  t.slots.clear();
  t.failed.clear();
  t.busy = false;
}

// Harvest every finished tick, in launch order among them (ticks hold
// disjoint slots and may finish out of order).
pa_status harvest(pa_server* s) {
  pa_server::Tick* fin[kTickPool];
  int nf = 0;
  for (auto& t : s->ticks) {
    if (!t.busy) continue;
    const cudaError_t q = cudaEventQuery(t.ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return scuda(s, q, "tick");
    fin[nf++] = &t;
  }
  std::sort(fin, fin + nf, [](const pa_server::Tick* a, const pa_server::Tick* b) {
    return a->seq < b->seq;
  });
  for (int k = 0; k < nf; ++k) finalize(s, *fin[k]);
  return PA_OK;
}

}  // namespace

extern "C" {

pa_status pa_server_create(const pa_config* base, int32_t generations, int32_t tick,
                           uint64_t budget_bytes, void* stream, pa_server** out) {
  pa::set_thread_error("");
  if (!out) return PA_EINVAL;
  *out = nullptr;
  if (!base || generations < 1 || tick < 1 || budget_bytes == 0) {
    pa::set_thread_error("base config, generations >= 1, tick >= 1 and a budget are required");
    return PA_EINVAL;
  }
  std::string why;
  if (!pa::config_ok(base, &why)) {
    pa::set_thread_error("base config: " + why);
    return PA_EINVAL;
  }
  if (base->islands >= 2) {
    pa::set_thread_error("the server runs one population per request (islands <= 1)");
    return PA_EUNSUPPORTED;
  }
  pa_server* s = new (std::nothrow) pa_server();
  if (!s) return PA_ENOMEM;
  s->base = *base;
  s->G = generations;
  s->tick = tick;
  s->budget = budget_bytes;
  if (stream) {
    s->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return PA_ECUDA;
    }
    s->own_stream = true;
  }
  // the tick pool's streams, events and first buffers now, not on a poll
  // (pinned allocations take milliseconds)
  for (auto& t : s->ticks) {
    pa_status st = tick_streams(s, t, 2);
    if (st == PA_OK) st = grow<void>(s, &t.d_seed_args, &t.h_seed_args, &t.seed_cap, 16 << 10);
    if (st == PA_OK) st = grow<void>(s, &t.d_solve_args, &t.h_solve_args, &t.solve_cap, 64 << 10);
    if (st == PA_OK) st = grow<int>(s, &t.d_counters, nullptr, &t.counters_cap, 256);
    if (st == PA_OK) st = grow<uint8_t>(s, nullptr, &t.h_best, &t.best_cap, 64 << 10);
    if (st == PA_OK) st = grow<double>(s, &t.d_bestfit, &t.h_bestfit, &t.fit_cap, 4 << 10);
    if (st == PA_OK && cudaMallocHost(&t.h_stage, (size_t)4 << 20) == cudaSuccess)
      t.stage_cap = (size_t)4 << 20;
    if (st != PA_OK) {
      pa::set_thread_error(s->err);
      destroy_server(s);
      return st;
    }
  }
  *out = s;
  return PA_OK;
}

void pa_server_destroy(pa_server* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  destroy_server(s);
}

const char* pa_server_last_error(const pa_server* s) { return s ? s->err.c_str() : ""; }

static pa_status submit_impl(pa_server* s, int64_t id, int32_t L, int32_t K, uint64_t seed,
                             const double* beta, const int32_t* user_xy_mm,
                             const int32_t* bs_xy_mm) {
  if (!beta || !user_xy_mm || !bs_xy_mm)
    return sfail(s, PA_EINVAL, "beta and positions are required");
  const pa_config c = slot_config(s, L, K);
  std::string why;
  if (!pa::config_ok(&c, &why)) return sfail(s, PA_EINVAL, "request: " + why);
  double bmax = 0.0;
  if (!pa::instance_ok(c, beta, user_xy_mm, bs_xy_mm, &bmax))
    return sfail(s, PA_EINVAL, "request: beta must be finite and > 0; positions within int32");
  if (!shape_runs(c))
    return sfail(s, PA_EUNSUPPORTED, "request shape does not fit the batched solve kernel");
  const size_t need = slot_bytes(c);
  if (need > s->budget)
    return sfail(s, PA_EBUSY, "one slot of this shape needs " + std::to_string(need) +
                                  " bytes; the budget is " + std::to_string(s->budget));
  pa_server::Req r;
  r.id = id;
  r.L = L;
  r.K = K;
  r.seed = seed;
  r.beta.assign(beta, beta + (size_t)L * L * K);
  r.uxy.assign(user_xy_mm, user_xy_mm + (size_t)2 * L * K);
  r.bxy.assign(bs_xy_mm, bs_xy_mm + (size_t)2 * L);
  s->pending.push_back(std::move(r));
  return PA_OK;
}

pa_status pa_server_submit(pa_server* s, int64_t id, int32_t L, int32_t K, uint64_t seed,
                           const double* beta, const int32_t* user_xy_mm,
                           const int32_t* bs_xy_mm) {
  if (!s) return PA_EINVAL;
  try {
    return submit_impl(s, id, L, K, seed, beta, user_xy_mm, bs_xy_mm);
  } catch (const std::bad_alloc&) {
    return sfail(s, PA_ENOMEM, "host memory for the request copy");
  } catch (...) {
    return sfail(s, PA_ENOMEM, "request copy failed");
  }
}

static pa_status tick_impl(pa_server* s);

pa_status pa_server_poll(pa_server* s, int32_t max_done, int64_t* done_ids, int32_t* done_status,
                         uint8_t* done_best, int64_t best_stride, double* done_fit,
                         int32_t* n_done, int32_t* n_active, int32_t* n_pending) {
  if (!s || !n_done) return PA_EINVAL;
  if (max_done < 0 || (done_best && best_stride < 0)) return sfail(s, PA_EINVAL, "bad outputs");
  *n_done = 0;
  pa_status st;
  try {
    st = harvest(s);
    if (st == PA_OK) st = tick_impl(s);
  } catch (const std::bad_alloc&) {
    st = sfail(s, PA_ENOMEM, "host memory during a tick");
  } catch (...) {
    st = sfail(s, PA_ENOMEM, "tick failed");
  }
  int nd = 0;
  while (nd < max_done && !s->done.empty()) {
    const pa_server::Done& d = s->done.front();
    if (done_ids) done_ids[nd] = d.id;
    if (done_status) done_status[nd] = d.st;
    if (done_best) std::memcpy(done_best + (int64_t)nd * best_stride, d.best.data(), d.best.size());
    if (done_fit) done_fit[nd] = d.fit;
    s->done.pop_front();
    ++nd;
  }
  *n_done = nd;
  if (n_active) {
    int a = 0;
    for (auto& sl : s->slots) a += sl.active ? 1 : 0;
    *n_active = a;
  }
  if (n_pending) *n_pending = (int32_t)s->pending.size();
  return st;
}

pa_status pa_server_wait(pa_server* s, int32_t timeout_us) {
  if (!s) return PA_EINVAL;
  pa_server::Tick* oldest = nullptr;
  for (auto& t : s->ticks)
    if (t.busy && (!oldest || t.seq < oldest->seq)) oldest = &t;
  if (!oldest) return PA_OK;
  if (timeout_us < 0) return scuda(s, cudaEventSynchronize(oldest->ev), "tick wait");
  const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  for (;;) {
    const cudaError_t q = cudaEventQuery(oldest->ev);
    if (q == cudaSuccess) return PA_OK;
    if (q != cudaErrorNotReady) return scuda(s, q, "tick");
    if (std::chrono::steady_clock::now() >= t_end) return PA_OK;
    std::this_thread::yield();
  }
}

pa_status pa_server_cancel(pa_server* s, int64_t id) {
  if (!s) return PA_EINVAL;
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
    if (it->id == id) {
      s->pending.erase(it);
      return PA_OK;
    }
  for (size_t i = 0; i < s->slots.size(); ++i) {
    pa_server::Slot& sl = s->slots[i];
    if (sl.ctx && sl.active && !sl.cancelled && sl.req == id) {
      if (sl.tick >= 0)
        sl.cancelled = true;  // released when its tick has finished
      else
        release(s, (int)i);
      return PA_OK;
    }
  }
  for (auto it = s->done.begin(); it != s->done.end(); ++it)
    if (it->id == id) {
      s->done.erase(it);
      return PA_OK;
    }
  return sfail(s, PA_EINVAL, "no queued, running or unreturned request has this id");
}

pa_status pa_server_inject_admission_failures(pa_server* s, int32_t count) {
  if (!s || count < 0) return PA_EINVAL;
  s->inject_failures = count;
  return PA_OK;
}

pa_status pa_server_stats(const pa_server* s, uint64_t* used_bytes, int32_t* n_slots,
                          int64_t* completed) {
  if (!s) return PA_EINVAL;
  if (used_bytes) *used_bytes = s->used;
  if (n_slots) {
    int n = 0;
    for (auto& sl : s->slots) n += sl.ctx ? 1 : 0;
    *n_slots = n;
  }
  if (completed) *completed = s->completed;
  return PA_OK;
}

}  // extern "C"

// Admission into free slots and one tick for every idle active slot, on a
// tick of the pool that is not in flight (none free: the next poll).
static pa_status tick_impl(pa_server* s) {
  pa_server::Tick* tp = nullptr;
  for (auto& t : s->ticks)
    if (!t.busy) {
      tp = &t;
      break;
    }
  if (!tp) return PA_OK;
  pa_server::Tick& t = *tp;
  pa_status st = tick_streams(s, t, 0);
  if (st != PA_OK) return st;
  if (t.dirty) {  // an earlier launch on this tick failed midway: let its work drain
    st = scuda(s, cudaStreamSynchronize(t.st), "tick drain");
    if (st != PA_OK) return st;
    t.dirty = false;
  }
  // pinned staging for this tick's admissions
  {
    size_t need = 0;
    for (const auto& r : s->pending) need += stage_bytes(r);
    need = std::min(need, (size_t)64 << 20);
    if (need > t.stage_cap) {  // doubling (4 MB at creation)
      const size_t cap = std::max({need, 2 * t.stage_cap, (size_t)16 << 20});
      cudaFreeHost(t.h_stage);
      t.h_stage = nullptr;
      t.stage_cap = 0;
      if (cudaMallocHost(&t.h_stage, cap) == cudaSuccess) t.stage_cap = cap;
      else (void)cudaGetLastError();
    }
    t.stage_used = 0;
  }
  // ---- admission, in arrival order
  int created_now = 0;
  std::vector<int> fresh;
  while (!s->pending.empty()) {
    pa_server::Req& r = s->pending.front();
    const auto key = std::make_pair(r.L, r.K);
    auto& fl = s->free_slots[key];
    const pa_config c = slot_config(s, r.L, r.K);
    int slot = -1;
    bool created = false;
    if (!fl.empty()) {
      slot = fl.back();
      fl.pop_back();
    } else {
      if (created_now == kMaxNewSlots) break;  // the next poll creates more
      const size_t need = slot_bytes(c);
      if (!make_room(s, need, key)) break;  // wait for running slots to finish
      ++created_now;
      pa_ctx* ctx = nullptr;
      pa_status cs;
      std::string why;
      if (s->inject_failures > 0) {
        --s->inject_failures;
        cs = PA_ECUDA;
        why = "injected admission failure";
      } else {
        cs = pa_create(&c, r.beta.data(), r.uxy.data(), r.bxy.data(), s->stream, &ctx);
        if (cs != PA_OK) why = pa_last_error(nullptr);
      }
      if (cs != PA_OK) {  // this request fails; the queue moves on
        s->err = "slot of request " + std::to_string(r.id) + ": " + why;
        complete(s, r.id, cs, r.L, r.K, nullptr, 0.0);
        s->pending.pop_front();
        continue;
      }
      for (size_t i = 0; i < s->slots.size() && slot < 0; ++i)
        if (!s->slots[i].ctx) slot = (int)i;
      if (slot < 0) {
        s->slots.emplace_back();
        slot = (int)s->slots.size() - 1;
      }
      prepare_variant(s, ctx);
      pa_server::Slot& ns = s->slots[slot];
      ns = pa_server::Slot();
      ns.ctx = ctx;
      ns.L = r.L;
      ns.K = r.K;
      ns.bytes = need;
      s->used += need;
      created = true;
    }
    pa_server::Slot& sl = s->slots[slot];
    sl.ctx->stream = t.st;
    sl.ctx->cfg.seed = r.seed;
    pa_status ls = PA_OK;
    if (!created && s->inject_failures > 0) {
      --s->inject_failures;
      ls = PA_ECUDA;
      s->err = "injected admission failure";
    } else if (!created) {  // pa_create uploaded a new slot's instance already
      const double* beta = r.beta.data();
      const int32_t* uxy = r.uxy.data();
      const int32_t* bxy = r.bxy.data();
      const size_t sb = stage_bytes(r);
      if (t.stage_used + sb <= t.stage_cap) {  // else the pageable copy (synchronous upload)
        unsigned char* h = t.h_stage + t.stage_used;
        const size_t nb = 8 * r.beta.size(), nu = 4 * r.uxy.size();
        const size_t ob = (nb + 15) & ~size_t(15), ou = (nu + 15) & ~size_t(15);
        std::memcpy(h, beta, nb);
        std::memcpy(h + ob, uxy, nu);
        std::memcpy(h + ob + ou, bxy, 4 * r.bxy.size());
        beta = reinterpret_cast<const double*>(h);
        uxy = reinterpret_cast<const int32_t*>(h + ob);
        bxy = reinterpret_cast<const int32_t*>(h + ob + ou);
        t.stage_used += sb;
      }
      t.dirty = true;  // uploads enqueued on the tick's stream
      ls = pa_load_instance(sl.ctx, beta, uxy, bxy);
      if (ls != PA_OK) s->err = pa_last_error(sl.ctx);
    }
    if (ls != PA_OK) {  // the slot stays usable for later requests
      sl.ctx->stream = s->stream;
      fl.push_back(slot);
      complete(s, r.id, ls, r.L, r.K, nullptr, 0.0);
      s->pending.pop_front();
      continue;
    }
    sl.req = r.id;
    sl.gen = 0;
    sl.active = true;
    sl.fresh = true;
    sl.cancelled = false;
    sl.ctx->cur = 0;
    fresh.push_back(slot);
    s->pending.pop_front();
  }
  // ---- the slots this tick advances: every active slot without a tick in flight
  std::map<std::tuple<int, int, int>, std::vector<int>> groups;
  int n_act = 0;
  for (size_t i = 0; i < s->slots.size(); ++i) {
    const auto& sl = s->slots[i];
    if (!sl.active || !sl.ctx) continue;
    ++n_act;
    if (sl.tick >= 0) continue;
    const pa_ctx* c = sl.ctx;
    groups[std::make_tuple(c->t32.NJ, c->t32.vec, c->cfg.prec)].push_back((int)i);
  }
  if (groups.empty()) return PA_OK;
  const int t_index = (int)(&t - s->ticks);
  // the tick waits for the slot creations and uploads on the server stream
  t.dirty = true;
  st = scuda(s, cudaEventRecord(t.fork, s->stream), "order");
  if (st == PA_OK) st = scuda(s, cudaStreamWaitEvent(t.st, t.fork, 0), "order wait");
  if (st != PA_OK) return st;
  // ---- seed the new slots (one launch)
  if (!fresh.empty()) {
    const size_t sb = pa::seed_args_bytes();
    st = grow<void>(s, &t.d_seed_args, &t.h_seed_args, &t.seed_cap, sb * fresh.size());
    if (st != PA_OK) return st;
    unsigned char* h = static_cast<unsigned char*>(t.h_seed_args);
    size_t smem = 0;
    const int sc = pa::seed_batch_cluster((int)fresh.size());
    for (size_t i = 0; i < fresh.size(); ++i)
      smem = std::max(smem, pa::seed_fill_args(s->slots[fresh[i]].ctx, h + sb * i, sc));
    st = scuda(s, cudaMemcpyAsync(t.d_seed_args, h, sb * fresh.size(), cudaMemcpyHostToDevice,
                                  t.st),
               "copy seed args");
    if (st == PA_OK)
      st = scuda(s, pa::launch_seed_batch(t.d_seed_args, (int)fresh.size(), smem, sc, t.st),
                 "seed kernel");
    if (st != PA_OK) return st;
  }
  // ---- one persistent launch per variant group, side by side
  size_t n_tick = 0;
  for (auto& kv : groups) n_tick += kv.second.size();
  const size_t ab = pa::solve_args_bytes();
  st = grow<void>(s, &t.d_solve_args, &t.h_solve_args, &t.solve_cap, ab * n_tick);
  if (st == PA_OK) st = grow<int>(s, &t.d_counters, nullptr, &t.counters_cap, sizeof(int) * groups.size());
  if (st == PA_OK) st = tick_streams(s, t, groups.size() > 1 ? groups.size() : 0);
  if (st != PA_OK) return st;
  t.slots.clear();
  t.g_now.clear();
  t.finish_k.clear();
  t.best_off.clear();
  t.failed.clear();
  int64_t best_total = 0;
  int n_fin = 0;
  for (auto& kv : groups)
    for (int i : kv.second) {
      const pa_server::Slot& sl = s->slots[i];
      const int g_now = std::min(s->tick, s->G - sl.gen);
      t.slots.push_back(i);
      t.g_now.push_back(g_now);
      if (sl.gen + g_now >= s->G) {
        t.finish_k.push_back(n_fin++);
        t.best_off.push_back(best_total);
        best_total += (int64_t)sl.L * sl.K;
      } else {
        t.finish_k.push_back(-1);
      }
    }
  st = grow<uint8_t>(s, nullptr, &t.h_best, &t.best_cap, (size_t)std::max<int64_t>(1, best_total));
  if (st == PA_OK)
    st = grow<double>(s, &t.d_bestfit, &t.h_bestfit, &t.fit_cap,
                      sizeof(double) * std::max(1, n_fin));
  if (st == PA_OK)
    st = scuda(s, cudaMemsetAsync(t.d_counters, 0, sizeof(int) * groups.size(), t.st),
               "reset counters");
  if (st != PA_OK) return st;
  std::map<int, size_t> pos_of;  // slot -> position in t.slots
  for (size_t m = 0; m < t.slots.size(); ++m) pos_of[t.slots[m]] = m;
  unsigned char* ha = static_cast<unsigned char*>(t.h_solve_args);
  size_t a_off = 0;
  int gk = 0;
  const bool forked = groups.size() > 1;
  if (forked) {
    st = scuda(s, cudaEventRecord(t.fork, t.st), "fork");
    if (st != PA_OK) return st;
  }
  for (auto& kv : groups) {
    const std::vector<int>& mem = kv.second;
    const pa_ctx* proto = s->slots[mem[0]].ctx;
    // cluster size: the largest that keeps every active slot resident at
    // once (16 CTAs for up to 9 slots on 152 SMs), smaller if it cannot fit;
    // while every active slot has 16 CTAs of its own, generations are
    // latency-bound: the one-instance kernel's column split, else the
    // throughput split
    int C = 16;
    while (C > 1 && n_act * C > proto->num_sms) C /= 2;
    bool latency = C == 16;
    size_t smem = 0;
    bool ok = false;
    for (; C >= 1 && !ok; C /= 2) {
      ok = true;
      smem = 0;
      for (size_t m = 0; m < mem.size(); ++m) {
        pa_server::Slot& sl = s->slots[mem[m]];
        const size_t p = pos_of[mem[m]];
        const int k = t.finish_k[p];
        uint8_t* best_row = k >= 0 ? sl.ctx->best_row : nullptr;
        double* best_fit = k >= 0 ? t.d_bestfit + k : nullptr;
        const size_t need = pa::solve_fill_args(sl.ctx, C, sl.gen, t.g_now[p],
                                                sl.ctx->pop[sl.ctx->cur],
                                                sl.ctx->pop[sl.ctx->cur ^ 1], sl.ctx->fit,
                                                best_row, best_fit, ha + a_off + ab * m, latency);
        if (need == 0) {
          ok = false;
          break;
        }
        smem = std::max(smem, need);
      }
      if (ok && pa::solve_batch_max_clusters(proto, C, smem, latency) < 1) ok = false;
      if (ok) break;
      if (latency) {  // the latency split does not fit: the throughput split, same C
        latency = false;
        C *= 2;
      }
    }
    if (!ok) {  // cannot happen for shapes checked at submit; fail these requests only
      for (int i : mem) {
        t.failed.push_back(i);
        t.g_now[pos_of[i]] = -1;
      }
      continue;
    }
    const int clusters =
        std::min<int>((int)mem.size(), pa::solve_batch_max_clusters(proto, C, smem, latency));
    unsigned char* dargs = static_cast<unsigned char*>(t.d_solve_args) + a_off;
    cudaStream_t gs = forked ? t.side[gk] : t.st;
    if (forked) st = scuda(s, cudaStreamWaitEvent(gs, t.fork, 0), "fork wait");
    if (st == PA_OK)
      st = scuda(s, cudaMemcpyAsync(dargs, ha + a_off, ab * mem.size(), cudaMemcpyHostToDevice,
                                    gs),
                 "copy solve args");
    if (st == PA_OK)
      st = scuda(s, pa::launch_solve_batch(proto, C, clusters, dargs, (int)mem.size(),
                                           t.d_counters + gk, smem, gs, latency),
                 "batched solve kernel");
    if (st == PA_OK && forked) st = scuda(s, cudaEventRecord(t.joined[gk], gs), "join");
    if (st != PA_OK) return st;
    a_off += ab * mem.size();
    ++gk;
  }
  if (forked)
    for (int k = 0; k < gk; ++k) {
      st = scuda(s, cudaStreamWaitEvent(t.st, t.joined[k], 0), "join wait");
      if (st != PA_OK) return st;
    }
  // ---- results of finishing slots to pinned memory
  for (size_t m = 0; m < t.slots.size(); ++m) {
    const int k = t.finish_k[m];
    if (k < 0) continue;
    const pa_server::Slot& sl = s->slots[t.slots[m]];
    st = scuda(s, cudaMemcpyAsync(t.h_best + t.best_off[k], sl.ctx->best_row, (size_t)sl.L * sl.K,
                                  cudaMemcpyDeviceToHost, t.st),
               "copy best");
    if (st != PA_OK) return st;
  }
  if (n_fin > 0) {
    st = scuda(s, cudaMemcpyAsync(t.h_bestfit, t.d_bestfit, sizeof(double) * n_fin,
                                  cudaMemcpyDeviceToHost, t.st),
               "copy best fit");
    if (st != PA_OK) return st;
  }
  st = scuda(s, cudaEventRecord(t.ev, t.st), "tick event");
  if (st != PA_OK) return st;
  for (int i : t.slots) s->slots[i].tick = t_index;
  for (int i : t.failed) s->slots[i].tick = t_index;
  t.busy = true;
  t.dirty = false;
  t.seq = ++s->tick_seq;
  return PA_OK;
}
