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
//   4. finished requests are copied back and returned; their slots free up.
// Requests that arrive while a tick runs join at the next tick, so work of
// many requests overlaps on the device.  A request's result is exactly what
// pa_solve gives for the same instance and seed alone: generations run in
// the same order with the same draws, whatever the tick length or the mix.
#include <algorithm>
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
}

struct pa_server {
  pa_config base{};
  int G = 0, tick = 0;
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  struct Slot {
    pa_ctx* ctx = nullptr;
    int L = 0, K = 0;
    int64_t req = -1;
    int gen = 0;
    bool active = false, fresh = false, done = false;
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
  cudaFree(s->d_bestfit);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // namespace

extern "C" {

pa_status pa_server_create(const pa_config* base, int32_t generations, int32_t tick,
                           uint64_t budget_bytes, void* stream, pa_server** out) {
  if (!out) return PA_EINVAL;
  *out = nullptr;
  if (!base || generations < 1 || tick < 1 || budget_bytes == 0) {
    pa::set_thread_error("base config, generations >= 1, tick >= 1 and a budget are required");
    return PA_EINVAL;
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

pa_status pa_server_submit(pa_server* s, int64_t id, int32_t L, int32_t K, uint64_t seed,
                           const double* beta, const int32_t* user_xy_mm,
                           const int32_t* bs_xy_mm) {
  if (!s) return PA_EINVAL;
  if (!beta || !user_xy_mm || !bs_xy_mm)
    return sfail(s, PA_EINVAL, "beta and positions are required");
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

pa_status pa_server_poll(pa_server* s, int32_t max_done, int64_t* done_ids, uint8_t* done_best,
                         int64_t best_stride, double* done_fit, int32_t* n_done,
                         int32_t* n_active, int32_t* n_pending) {
  if (!s || !n_done) return PA_EINVAL;
  *n_done = 0;
  pa_status st = PA_OK;
  // ---- 1. admission
  std::vector<int> fresh;
  while (!s->pending.empty()) {
    pa_server::Req& r = s->pending.front();
    auto key = std::make_pair(r.L, r.K);
    auto& fl = s->free_slots[key];
    int slot = -1;
    if (!fl.empty()) {
      slot = fl.back();
      fl.pop_back();
    } else {
      pa_config c = s->base;
      c.L = r.L;
      c.K = r.K;
      c.tau_p = r.K;
      c.kmeans_k = r.K;
      const size_t need = slot_bytes(c);
      if (s->used + need > s->budget) break;  // wait for memory to free up
      pa_ctx* ctx = nullptr;
      st = pa_create(&c, r.beta.data(), r.uxy.data(), r.bxy.data(), s->stream, &ctx);
      if (st != PA_OK) return sfail(s, st, std::string("slot: ") + pa_last_error(nullptr));
      pa_server::Slot sl;
      sl.ctx = ctx;
      sl.L = r.L;
      sl.K = r.K;
      s->slots.push_back(sl);
      slot = (int)s->slots.size() - 1;
      s->used += need;
    }
    pa_server::Slot& sl = s->slots[slot];
    sl.ctx->cfg.seed = r.seed;
    st = pa_load_instance(sl.ctx, r.beta.data(), r.uxy.data(), r.bxy.data());
    if (st != PA_OK) return sfail(s, st, pa_last_error(sl.ctx));
    sl.req = r.id;
    sl.gen = 0;
    sl.active = true;
    sl.fresh = true;
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
    if (!sl.active) continue;
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
  {
    size_t fcap_before = s->fit_cap;
    st = grow<double>(s, &s->d_bestfit, &s->h_bestfit, &s->fit_cap,
                      sizeof(double) * std::max<size_t>(1, finishing.size()), true);
    (void)fcap_before;
    if (st != PA_OK) return st;
  }
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
                                                best_fit, ha + a_off + ab * m);
        if (need == 0) {
          ok = false;
          break;
        }
        smem = std::max(smem, need);
      }
      if (ok && pa::solve_batch_max_clusters(proto, C, smem) < 1) ok = false;
      if (ok) break;
    }
    if (!ok) return sfail(s, PA_EUNSUPPORTED, "request shape does not fit the solve kernel");
    const int clusters =
        std::min<int>((int)mem.size(), pa::solve_batch_max_clusters(proto, C, smem));
    unsigned char* dargs = static_cast<unsigned char*>(s->d_solve_args) + a_off;
    st = scuda(s, cudaMemcpyAsync(dargs, ha + a_off, ab * mem.size(), cudaMemcpyHostToDevice,
                                  s->stream),
               "copy solve args");
    // the variants' launches run side by side: group k on side stream k,
    // forked from and joined back into the server stream
    if (st == PA_OK) st = side_stream(s, gk);
    if (st == PA_OK) st = scuda(s, cudaEventRecord(s->fork, s->stream), "fork");
    if (st == PA_OK) st = scuda(s, cudaStreamWaitEvent(s->side[gk], s->fork, 0), "fork wait");
    if (st == PA_OK)
      st = scuda(s, pa::launch_solve_batch(proto, C, clusters, dargs, (int)mem.size(),
                                           s->d_counters + gk, smem, s->side[gk]),
                 "batched solve kernel");
    if (st == PA_OK) st = scuda(s, cudaEventRecord(s->joined[gk], s->side[gk]), "join");
    if (st != PA_OK) return st;
    a_off += ab * mem.size();
    ++gk;
  }
  for (int k = 0; k < gk; ++k) {
    st = scuda(s, cudaStreamWaitEvent(s->stream, s->joined[k], 0), "join wait");
    if (st != PA_OK) return st;
  }
  // ---- 4. collect finished requests
  for (int i : finishing) {
    pa_server::Slot& sl = s->slots[i];
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
  for (auto& kv : groups)
    for (int i : kv.second) {
      pa_server::Slot& sl = s->slots[i];
      const int g_now = std::min(s->tick, s->G - sl.gen);
      sl.gen += g_now;
      sl.ctx->cur ^= 1;
      sl.ctx->generation = sl.gen;
    }
  int nd = 0;
  for (size_t k = 0; k < finishing.size(); ++k) {
    pa_server::Slot& sl = s->slots[finishing[k]];
    if (nd < max_done) {
      if (done_ids) done_ids[nd] = sl.req;
      if (done_best)
        std::memcpy(done_best + (int64_t)nd * best_stride, s->h_best + sl.best_off,
                    (size_t)sl.L * sl.K);
      if (done_fit) done_fit[nd] = s->h_bestfit[k];
      ++nd;
    }
    sl.active = false;
    sl.req = -1;
    s->free_slots[std::make_pair(sl.L, sl.K)].push_back(finishing[k]);
    ++s->completed;
  }
  *n_done = nd;
  if (n_active) {
    int a = 0;
    for (auto& sl : s->slots) a += sl.active ? 1 : 0;
    *n_active = a;
  }
  if (n_pending) *n_pending = (int32_t)s->pending.size();
  return PA_OK;
}

pa_status pa_server_stats(const pa_server* s, uint64_t* used_bytes, int32_t* n_slots,
                          int64_t* completed) {
  if (!s) return PA_EINVAL;
  if (used_bytes) *used_bytes = s->used;
  if (n_slots) *n_slots = (int32_t)s->slots.size();
  if (completed) *completed = s->completed;
  return PA_OK;
}

}  // extern "C"
