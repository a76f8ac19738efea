// pa_server.cu -- continuous-batching solve server.
//
// Requests (one pilot-assignment instance each: L, K, gains, positions,
// seed) arrive at any time through pa_server_submit.  Each pa_server_poll
// runs one scheduling tick:
//   1. admission: queued requests take free slots of their (L, K) class --
//      a slot is a resident context (gains, tables, double-buffered
//      population on the GPU); new slots are created while the device
//      memory they need stays within the server's budget;
//   2. the newly admitted slots are seeded in one batched launch;
//   3. every active slot advances by up to `tick` generations in one
//      persistent batched solve launch per kernel variant (populations stay
//      resident between ticks; a slot reaching G generations also gets its
//      final evaluation and best member);
//   4. finished requests are copied back into a completion queue that
//      polls drain (up to the caller's max_done per poll); their slots
//      stay resident for the next request of the same class.
// Requests that arrive while a tick runs join at the next tick, so work of
// many requests overlaps on the device.  A request's result is exactly what
// pa_solve gives for the same instance and seed alone: generations run in
// the same order with the same draws, whatever the tick length or the mix.
//
// Liveness: requests are checked at submit (shape, values, a slot of its
// shape within the budget), so every queued request can eventually be
// admitted; when the head of the queue needs memory, idle slots (of other
// classes first) are destroyed; an admission that fails anyway completes
// that request with the error and the queue moves on.  No C++ exception
// crosses the C ABI: allocation failures return PA_ENOMEM.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "pa_internal.cuh"

namespace pa {
void set_thread_error(const std::string& msg);
bool config_ok(const pa_config* c, std::string* why);
void f32_geometry(int L, int K, int* NJ, int* RS, int* vec);
}

struct pa_server {
  pa_config base{};
  int G = 0, tick = 0;
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  struct Slot {
    pa_ctx* ctx = nullptr;  // null: destroyed (entry reusable)
    int L = 0, K = 0;
    size_t bytes = 0;       // device bytes charged to the budget
    int64_t req = -1;
    int gen = 0;
    bool active = false, fresh = false, failed = false;
    int64_t best_off = 0;  // offset in the pinned results buffer
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
  // pinned staging of the requests admitted in one tick (their uploads are
  // asynchronous; the tick's final synchronisation ends them)
  unsigned char* h_stage = nullptr;
  size_t stage_cap = 0, stage_used = 0;
  bool stage_busy = false;  // uploads from the staging buffer may be in flight
  // per-tick device/pinned scratch
  void* d_seed_args = nullptr;
  void* h_seed_args = nullptr;
  size_t seed_cap = 0;
  void* d_solve_args = nullptr;
  void* h_solve_args = nullptr;
  size_t solve_cap = 0;
  int* d_counters = nullptr;
  int counters_cap = 0;
  uint8_t* h_best = nullptr;  // pinned: best rows of finishing slots
  double* h_bestfit = nullptr;
  double* d_bestfit = nullptr;
  size_t best_cap = 0, fit_cap = 0;
  // side streams of the variant groups of a tick, with their events
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> joined;
  cudaEvent_t fork = nullptr;
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

template <typename T>
pa_status grow(pa_server* s, T** dev, T** host, size_t* cap, size_t need, bool pinned_host) {
  if (need <= *cap) return PA_OK;
  size_t n = std::max(need, *cap * 2 + 64);
  if (dev) {
    cudaFree(*dev);
    *dev = nullptr;
    pa_status st = scuda(s, cudaMalloc(dev, n), "cudaMalloc server scratch");
    if (st != PA_OK) return st;
  }
  if (host) {
    if (pinned_host) cudaFreeHost(*host);
    *host = nullptr;
    pa_status st = scuda(s, cudaMallocHost(host, n), "cudaMallocHost server scratch");
    if (st != PA_OK) return st;
  }
  *cap = n;
  return PA_OK;
}

// Side stream k (created on first use).
pa_status side_stream(pa_server* s, int k) {
  if (!s->fork) {
    pa_status st = scuda(s, cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming), "event");
    if (st != PA_OK) return st;
  }
  while ((int)s->side.size() <= k) {
    cudaStream_t x = nullptr;
    cudaEvent_t e = nullptr;
    pa_status st = scuda(s, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "stream");
    if (st != PA_OK) return st;
    st = scuda(s, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    if (st != PA_OK) {
      cudaStreamDestroy(x);
      return st;
    }
    s->side.push_back(x);
    s->joined.push_back(e);
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
  for (auto x : s->side) cudaStreamDestroy(x);
  for (auto e : s->joined) cudaEventDestroy(e);
  if (s->fork) cudaEventDestroy(s->fork);
  for (auto& sl : s->slots) pa_destroy(sl.ctx);
  cudaFree(s->d_seed_args);
  cudaFreeHost(s->h_seed_args);
  cudaFree(s->d_solve_args);
  cudaFreeHost(s->h_solve_args);
  cudaFree(s->d_counters);
  cudaFreeHost(s->h_best);
  cudaFreeHost(s->h_bestfit);
  cudaFreeHost(s->h_stage);
  cudaFree(s->d_bestfit);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
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
    st = tick_impl(s);
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

pa_status pa_server_cancel(pa_server* s, int64_t id) {
  if (!s) return PA_EINVAL;
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
    if (it->id == id) {
      s->pending.erase(it);
      return PA_OK;
    }
  for (size_t i = 0; i < s->slots.size(); ++i) {
    pa_server::Slot& sl = s->slots[i];
    if (sl.ctx && sl.active && sl.req == id) {
      sl.active = false;
      sl.fresh = false;
      sl.req = -1;
      s->free_slots[std::make_pair(sl.L, sl.K)].push_back((int)i);
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

}  // extern "C"

// Bytes of pinned staging for one request's upload, 16-byte aligned parts.
static size_t stage_bytes(const pa_server::Req& r) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  return al(8 * r.beta.size()) + al(4 * r.uxy.size()) + al(4 * r.bxy.size());
}

static pa_status tick_impl(pa_server* s) {
  pa_status st = PA_OK;
  // pinned staging for this tick's admissions (grown between ticks only:
  // earlier uploads of this tick may still read the old buffer otherwise;
  // a tick that failed before its final synchronisation may have left
  // uploads in flight)
  if (s->stage_busy) {
    st = scuda(s, cudaStreamSynchronize(s->stream), "staging sync");
    if (st != PA_OK) return st;
    s->stage_busy = false;
  }
  {
    size_t need = 0;
    for (const auto& r : s->pending) need += stage_bytes(r);
    need = std::min(need, (size_t)64 << 20);
    if (need > s->stage_cap) {  // rare: 4 MB first, then doubling (pinned allocations are slow)
      const size_t cap = std::max({need, 2 * s->stage_cap, (size_t)16 << 20});
      cudaFreeHost(s->h_stage);
      s->h_stage = nullptr;
      s->stage_cap = 0;
      if (cudaMallocHost(&s->h_stage, cap) == cudaSuccess) s->stage_cap = cap;
      else (void)cudaGetLastError();
    }
    s->stage_used = 0;
  }
  // ---- 1. admission, in arrival order; at most kMaxNewSlots contexts are
  // created per tick (creating one allocates and synchronises), so a burst
  // of new classes or a backlog cannot stall one tick for everyone
  constexpr int kMaxNewSlots = 4;
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
      if (created_now == kMaxNewSlots) break;  // the next tick creates more
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
    pa_status ls = PA_OK;
    if (created) {  // pa_create uploaded this request's instance already
      sl.ctx->cfg.seed = r.seed;
    } else if (s->inject_failures > 0) {
      --s->inject_failures;
      ls = PA_ECUDA;
      s->err = "injected admission failure";
    } else {
      sl.ctx->cfg.seed = r.seed;
      const double* beta = r.beta.data();
      const int32_t* uxy = r.uxy.data();
      const int32_t* bxy = r.bxy.data();
      const size_t sb = stage_bytes(r);
      if (s->stage_used + sb <= s->stage_cap) {  // else the pageable copy (synchronous upload)
        unsigned char* h = s->h_stage + s->stage_used;
        const size_t nb = 8 * r.beta.size(), nu = 4 * r.uxy.size();
        std::memcpy(h, beta, nb);
        std::memcpy(h + ((nb + 15) & ~size_t(15)), uxy, nu);
        std::memcpy(h + ((nb + 15) & ~size_t(15)) + ((nu + 15) & ~size_t(15)), bxy,
                    4 * r.bxy.size());
        beta = reinterpret_cast<const double*>(h);
        uxy = reinterpret_cast<const int32_t*>(h + ((nb + 15) & ~size_t(15)));
        bxy = reinterpret_cast<const int32_t*>(h + ((nb + 15) & ~size_t(15)) +
                                               ((nu + 15) & ~size_t(15)));
        s->stage_used += sb;
        s->stage_busy = true;
      }
      ls = pa_load_instance(sl.ctx, beta, uxy, bxy);
      if (ls != PA_OK) s->err = pa_last_error(sl.ctx);
    }
    if (ls != PA_OK) {  // the slot stays usable for later requests
      fl.push_back(slot);
      complete(s, r.id, ls, r.L, r.K, nullptr, 0.0);
      s->pending.pop_front();
      continue;
    }
    sl.req = r.id;
    sl.gen = 0;
    sl.active = true;
    sl.fresh = true;
    sl.failed = false;
    sl.ctx->cur = 0;
    fresh.push_back(slot);
    s->pending.pop_front();
  }
  // ---- 2. seed the new slots
  if (!fresh.empty()) {
    const size_t sb = pa::seed_args_bytes();
    unsigned char* h = nullptr;
    st = grow<void>(s, &s->d_seed_args, &s->h_seed_args, &s->seed_cap, sb * fresh.size(), true);
    if (st != PA_OK) return st;
    h = static_cast<unsigned char*>(s->h_seed_args);
    size_t smem = 0;
    const int sc = pa::seed_batch_cluster((int)fresh.size());
    for (size_t i = 0; i < fresh.size(); ++i)
      smem = std::max(smem, pa::seed_fill_args(s->slots[fresh[i]].ctx, h + sb * i, sc));
    st = scuda(s, cudaMemcpyAsync(s->d_seed_args, h, sb * fresh.size(), cudaMemcpyHostToDevice,
                                  s->stream),
               "copy seed args");
    if (st == PA_OK)
      st = scuda(s, pa::launch_seed_batch(s->d_seed_args, (int)fresh.size(), smem, sc, s->stream),
                 "seed kernel");
    if (st != PA_OK) return st;
    for (int i : fresh) s->slots[i].fresh = false;
  }
  // ---- 3. one tick of generations for every active slot, grouped by variant
  std::map<std::tuple<int, int, int>, std::vector<int>> groups;
  int n_act = 0;
  for (size_t i = 0; i < s->slots.size(); ++i) {
    const auto& sl = s->slots[i];
    if (!sl.active || !sl.ctx) continue;
    ++n_act;
    const pa_ctx* c = sl.ctx;
    groups[std::make_tuple(c->t32.NJ, c->t32.vec, c->cfg.prec)].push_back((int)i);
  }
  const size_t ab = pa::solve_args_bytes();
  st = grow<void>(s, &s->d_solve_args, &s->h_solve_args, &s->solve_cap, ab * std::max(1, n_act),
                  true);
  if (st != PA_OK) return st;
  if (s->counters_cap < (int)groups.size()) {
    cudaFree(s->d_counters);
    s->d_counters = nullptr;
    st = scuda(s, cudaMalloc(&s->d_counters, sizeof(int) * std::max<size_t>(1, groups.size())),
               "cudaMalloc counters");
    if (st != PA_OK) return st;
    s->counters_cap = (int)groups.size();
  }
  // results of slots finishing this tick: rows in a pinned buffer, fitness
  // through a device array
  std::vector<int> finishing;
  int64_t best_total = 0;
  for (auto& kv : groups)
    for (int i : kv.second)
      if (s->slots[i].gen + s->tick >= s->G) {
        finishing.push_back(i);
        s->slots[i].best_off = best_total;
        best_total += (int64_t)s->slots[i].L * s->slots[i].K;
      }
  st = grow<uint8_t>(s, nullptr, &s->h_best, &s->best_cap, std::max<int64_t>(1, best_total), true);
  if (st != PA_OK) return st;
  st = grow<double>(s, &s->d_bestfit, &s->h_bestfit, &s->fit_cap,
                    sizeof(double) * std::max<size_t>(1, finishing.size()), true);
  if (st != PA_OK) return st;
  std::map<int, int> fin_index;
  for (size_t k = 0; k < finishing.size(); ++k) fin_index[finishing[k]] = (int)k;
  if (!groups.empty()) {
    st = scuda(s, cudaMemsetAsync(s->d_counters, 0, sizeof(int) * groups.size(), s->stream),
               "reset counters");
    if (st != PA_OK) return st;
  }
  unsigned char* ha = static_cast<unsigned char*>(s->h_solve_args);
  size_t a_off = 0;
  int gk = 0;
  for (auto& kv : groups) {
    const std::vector<int>& mem = kv.second;
    const pa_ctx* proto = s->slots[mem[0]].ctx;
    // cluster size: the largest that keeps every active slot resident at
    // once (16 CTAs for up to 9 slots on 152 SMs), smaller if it cannot fit
    int C = 16;
    while (C > 1 && n_act * C > proto->num_sms) C /= 2;
    // while every active slot has 16 CTAs of its own, generations are
    // latency-bound: the one-instance kernel's column split, else the
    // throughput split
    bool latency = C == 16;
    size_t smem = 0;
    bool ok = false;
    for (; C >= 1 && !ok; C /= 2) {
      ok = true;
      smem = 0;
      for (size_t m = 0; m < mem.size(); ++m) {
        pa_server::Slot& sl = s->slots[mem[m]];
        const int g_now = std::min(s->tick, s->G - sl.gen);
        const bool fin = sl.gen + g_now >= s->G;
        uint8_t* best_row = fin ? sl.ctx->best_row : nullptr;
        double* best_fit = fin ? s->d_bestfit + fin_index[mem[m]] : nullptr;
        const size_t need = pa::solve_fill_args(sl.ctx, C, sl.gen, g_now, sl.ctx->pop[sl.ctx->cur],
                                                sl.ctx->pop[sl.ctx->cur ^ 1], sl.ctx->fit, best_row,
                                                best_fit, ha + a_off + ab * m, latency);
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
      for (int i : mem) s->slots[i].failed = true;
      continue;
    }
    const int clusters =
        std::min<int>((int)mem.size(), pa::solve_batch_max_clusters(proto, C, smem, latency));
    unsigned char* dargs = static_cast<unsigned char*>(s->d_solve_args) + a_off;
    st = scuda(s, cudaMemcpyAsync(dargs, ha + a_off, ab * mem.size(), cudaMemcpyHostToDevice,
                                  s->stream),
               "copy solve args");
    // one group runs on the server stream itself; several run side by side,
    // group k on side stream k, forked from and joined back into it
    const bool forked = groups.size() > 1;
    if (st == PA_OK && forked) st = side_stream(s, gk);
    if (st == PA_OK && forked) st = scuda(s, cudaEventRecord(s->fork, s->stream), "fork");
    if (st == PA_OK && forked)
      st = scuda(s, cudaStreamWaitEvent(s->side[gk], s->fork, 0), "fork wait");
    if (st == PA_OK)
      st = scuda(s, pa::launch_solve_batch(proto, C, clusters, dargs, (int)mem.size(),
                                           s->d_counters + gk, smem,
                                           forked ? s->side[gk] : s->stream, latency),
                 "batched solve kernel");
    if (st == PA_OK && forked) st = scuda(s, cudaEventRecord(s->joined[gk], s->side[gk]), "join");
    if (st != PA_OK) return st;
    a_off += ab * mem.size();
    ++gk;
  }
  if (groups.size() > 1)
    for (int k = 0; k < gk; ++k) {
      st = scuda(s, cudaStreamWaitEvent(s->stream, s->joined[k], 0), "join wait");
      if (st != PA_OK) return st;
    }
  // ---- 4. collect finished requests
  for (int i : finishing) {
    pa_server::Slot& sl = s->slots[i];
    if (sl.failed) continue;
    st = scuda(s, cudaMemcpyAsync(s->h_best + sl.best_off, sl.ctx->best_row,
                                  (size_t)sl.L * sl.K, cudaMemcpyDeviceToHost, s->stream),
               "copy best");
    if (st != PA_OK) return st;
  }
  if (!finishing.empty()) {
    st = scuda(s, cudaMemcpyAsync(s->h_bestfit, s->d_bestfit, sizeof(double) * finishing.size(),
                                  cudaMemcpyDeviceToHost, s->stream),
               "copy best fit");
    if (st != PA_OK) return st;
  }
  st = scuda(s, cudaStreamSynchronize(s->stream), "tick sync");
  if (st != PA_OK) return st;
  s->stage_busy = false;
  for (auto& kv : groups)
    for (int i : kv.second) {
      pa_server::Slot& sl = s->slots[i];
      if (sl.failed) {  // released without a result
        complete(s, sl.req, PA_EUNSUPPORTED, sl.L, sl.K, nullptr, 0.0);
        sl.active = false;
        sl.failed = false;
        sl.req = -1;
        s->free_slots[std::make_pair(sl.L, sl.K)].push_back(i);
        continue;
      }
      const int g_now = std::min(s->tick, s->G - sl.gen);
      sl.gen += g_now;
      sl.ctx->cur ^= 1;
      sl.ctx->generation = sl.gen;
    }
  for (size_t k = 0; k < finishing.size(); ++k) {
    pa_server::Slot& sl = s->slots[finishing[k]];
    if (!sl.active) continue;  // failed above
    complete(s, sl.req, PA_OK, sl.L, sl.K, s->h_best + sl.best_off, s->h_bestfit[k]);
    sl.active = false;
    sl.req = -1;
    s->free_slots[std::make_pair(sl.L, sl.K)].push_back(finishing[k]);
  }
  return PA_OK;
}

extern "C" {

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
