// pa_batch.cu -- many independent pilot-assignment instances of uneven size
// solved together (the batched form of the Alg. 1 loop).
//
// Instances are grouped by kernel variant (precision, SINR mode, BS-column
// width NJ, load width); each group runs as ONE persistent launch of
// k_solve_batch in which every thread-block cluster takes the next instance
// from a counter until the group is done, so uneven instances balance
// across the GPU.  Seeding of all instances is one launch (a cluster of
// CTAs per instance, 16 while the batch stays resident, down to 1).  The
// whole batch solve -- counter reset, seeding, the group
// launches on parallel streams, and the copies of the best members to the
// host -- is captured once into a CUDA graph and replayed.  The tiling of
// each group -- CTA size (1024 threads, one CTA per SM, or 256, four per SM
// and so several instances sharing an SM) and cluster size (1 to 16 CTAs
// per instance) -- is picked by pa_batch_tune, which times the candidates
// on the batch itself; the results do not depend on it (every instance's
// arithmetic is the same whatever the tiling).
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "pa_internal.cuh"

namespace pa {
void set_thread_error(const std::string& msg);
}

struct pa_batch {
  int n = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<pa_ctx*> ctx;
  struct Group {
    std::vector<int> members;
    int C = 0;
    int threads = 1024;  // CTA size: 1024 (one CTA per SM) or 256 (four per SM)
    bool latency = false;  // 1024-thread CTAs with the one-instance column split
    int cap8 = 8;  // resident clusters: cap8/8 of what fits (the rest of the GPU for the others)
    int clusters = 0;
    size_t smem = 0;
    std::vector<unsigned char> h_args;
    void* d_args = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Group> groups;
  void* d_seed_args = nullptr;
  size_t seed_smem = 0;
  int seed_C = 1;  // cluster size of the batched seeding launch
  int* d_counters = nullptr;
  uint8_t* d_best = nullptr;
  double* d_bestfit = nullptr;
  uint8_t* h_best = nullptr;     // pinned
  double* h_bestfit = nullptr;   // pinned
  std::vector<int64_t> best_off;
  int64_t best_bytes = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_G = -1;
  cudaEvent_t fork = nullptr;
  bool own_stream = false;
  unsigned long long* d_stamp = nullptr;  // [n] completion of each instance, [n] start (ns)
  std::string err;
};

namespace {

// The start of a batch solve on the device clock (ns).
__global__ void k_stamp(unsigned long long* p) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *p = t;
}

pa_status bfail(pa_batch* b, pa_status st, const std::string& m) {
  if (b) b->err = m;
  return st;
}

pa_status bcuda(pa_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PA_OK;
  return bfail(b, e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

void destroy_batch(pa_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& g : b->groups) {
    cudaFree(g.d_args);
    if (g.side) cudaStreamDestroy(g.side);
    if (g.done) cudaEventDestroy(g.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  cudaFree(b->d_seed_args);
  cudaFree(b->d_counters);
  cudaFree(b->d_stamp);
  cudaFree(b->d_best);
  cudaFree(b->d_bestfit);
  cudaFreeHost(b->h_best);
  cudaFreeHost(b->h_bestfit);
  for (pa_ctx* c : b->ctx) pa_destroy(c);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

// (Re)build one group's argument records for cluster size C and G
// generations; 0 on success, else the status.
pa_status build_group_args(pa_batch* b, pa_batch::Group& g, int C, int G, int threads,
                           bool latency) {
  const size_t ab = pa::solve_args_bytes();
  std::vector<unsigned char> h(ab * g.members.size());
  size_t smem = 0;
  for (size_t m = 0; m < g.members.size(); ++m) {
    const int i = g.members[m];
    pa_ctx* c = b->ctx[i];
    const size_t s = pa::solve_fill_args(c, C, 0, G, c->pop[0], c->pop[1], c->fit,
                                         b->d_best + b->best_off[i], b->d_bestfit + i,
                                         h.data() + m * ab, latency, threads);
    if (s == 0) return PA_EUNSUPPORTED;
    pa::solve_args_set_stamp(h.data() + m * ab, b->d_stamp + i);
    smem = std::max(smem, s);
  }
  const int maxc = pa::solve_batch_max_clusters(b->ctx[g.members[0]], C, smem, latency, threads);
  if (maxc < 1) return PA_EUNSUPPORTED;
  if (!g.d_args) {
    pa_status st = bcuda(b, cudaMalloc(&g.d_args, h.size()), "cudaMalloc batch args");
    if (st != PA_OK) return st;
  }
  pa_status st = bcuda(b, cudaMemcpy(g.d_args, h.data(), h.size(), cudaMemcpyHostToDevice),
                       "copy batch args");
  if (st != PA_OK) return st;
  g.h_args.swap(h);
  g.C = C;
  g.threads = threads;
  g.latency = latency;
  g.smem = smem;
  g.clusters = std::min<int>((int)g.members.size(), std::max(1, maxc * g.cap8 / 8));
  return PA_OK;
}

// Cluster size with the fewest CTAs that still gives every SM work, as the
// starting point before tuning.
int default_cluster(const pa_batch* b, const pa_batch::Group& g) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  int C = 1;
  while (C < 16 && (int)g.members.size() * C < sms) C *= 2;
  return C;
}

pa_status run_groups(pa_batch* b, cudaStream_t st) {
  k_stamp<<<1, 1, 0, st>>>(b->d_stamp + b->n);
  pa::count_launch();
  pa_status s = bcuda(b, cudaGetLastError(), "stamp kernel");
  if (s != PA_OK) return s;
  s = bcuda(b, cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->groups.size(), st),
            "reset counters");
  if (s != PA_OK) return s;
  s = bcuda(b, pa::launch_seed_batch(b->d_seed_args, b->n, b->seed_smem, b->seed_C, st),
            "seed kernel");
  if (s != PA_OK) return s;
  s = bcuda(b, cudaEventRecord(b->fork, st), "fork");
  if (s != PA_OK) return s;
  for (size_t k = 0; k < b->groups.size(); ++k) {
    auto& g = b->groups[k];
    s = bcuda(b, cudaStreamWaitEvent(g.side, b->fork, 0), "fork wait");
    if (s != PA_OK) return s;
    s = bcuda(b, pa::launch_solve_batch(b->ctx[g.members[0]], g.C, g.clusters, g.d_args,
                                        (int)g.members.size(), b->d_counters + k, g.smem, g.side,
                                        g.latency, g.threads),
              "batched solve kernel");
    if (s != PA_OK) return s;
    s = bcuda(b, cudaEventRecord(g.done, g.side), "join");
    if (s != PA_OK) return s;
    s = bcuda(b, cudaStreamWaitEvent(st, g.done, 0), "join wait");
    if (s != PA_OK) return s;
  }
  return PA_OK;
}

}  // namespace

extern "C" {

pa_status pa_batch_create(int32_t n, const pa_config* cfgs, const double* const* betas,
                          const int32_t* const* user_xy_mm, const int32_t* const* bs_xy_mm,
                          void* stream, pa_batch** out) {
  pa::set_thread_error("");
  if (!out) return PA_EINVAL;
  *out = nullptr;
  if (n < 1 || !cfgs || !betas) {
    pa::set_thread_error("n >= 1, cfgs and betas are required");
    return PA_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (cfgs[i].islands >= 2) {
      pa::set_thread_error("instance " + std::to_string(i) +
                           ": batches run one population per instance (islands <= 1)");
      return PA_EUNSUPPORTED;
    }
  pa_batch* b = new (std::nothrow) pa_batch();
  if (!b) return PA_ENOMEM;
  b->n = n;
  cudaGetDevice(&b->device);
  // graphs cannot be captured on the legacy default stream: without a
  // caller stream the batch uses a stream of its own
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return PA_ECUDA;
    }
    b->own_stream = true;
  }
  stream = b->stream;
  pa_status st = PA_OK;
  b->ctx.assign(n, nullptr);
  b->best_off.assign(n, 0);
  for (int i = 0; i < n && st == PA_OK; ++i) {
    const int32_t* u = user_xy_mm ? user_xy_mm[i] : nullptr;
    const int32_t* s = bs_xy_mm ? bs_xy_mm[i] : nullptr;
    st = pa_create(&cfgs[i], betas[i], u, s, stream, &b->ctx[i]);
    if (st != PA_OK) {
      b->err = std::string("instance ") + std::to_string(i) + ": " + pa_last_error(nullptr);
      break;
    }
    b->best_off[i] = b->best_bytes;
    b->best_bytes += (int64_t)cfgs[i].L * cfgs[i].K;
  }
  // kernel-variant groups
  std::map<std::tuple<int, int, int, int>, int> key2g;
  if (st == PA_OK) {
    for (int i = 0; i < n; ++i) {
      const pa_ctx* c = b->ctx[i];
      const auto key = std::make_tuple(c->cfg.prec, c->cfg.mode,
                                       c->cfg.prec == PA_FP32 ? c->t32.NJ : 0,
                                       c->cfg.prec == PA_FP32 ? c->t32.vec : 0);
      auto it = key2g.find(key);
      if (it == key2g.end()) {
        key2g[key] = (int)b->groups.size();
        b->groups.emplace_back();
        b->groups.back().members.push_back(i);
      } else {
        b->groups[it->second].members.push_back(i);
      }
    }
    // longest first: each group's queue in decreasing work (N L^2 K gathers
    // per generation), so the last instances a cluster takes are short ones;
    // the heaviest group is launched first
    auto work = [&](int i) {
      const pa_config& c = b->ctx[i]->cfg;
      return (int64_t)c.N * c.L * c.L * c.K;
    };
    for (auto& g : b->groups)
      std::stable_sort(g.members.begin(), g.members.end(),
                       [&](int x, int y) { return work(x) > work(y); });
    auto gwork = [&](const pa_batch::Group& g) {
      int64_t w = 0;
      for (int i : g.members) w += work(i);
      return w;
    };
    std::stable_sort(b->groups.begin(), b->groups.end(),
                     [&](const pa_batch::Group& x, const pa_batch::Group& y) {
                       return gwork(x) > gwork(y);
                     });
  }
  auto chk = [&](cudaError_t e, const char* what) {
    if (st == PA_OK) st = bcuda(b, e, what);
    return st == PA_OK;
  };
  if (st == PA_OK) {
    chk(cudaMalloc(&b->d_best, std::max<int64_t>(1, b->best_bytes)), "cudaMalloc best");
    chk(cudaMalloc(&b->d_bestfit, sizeof(double) * n), "cudaMalloc best fit");
    chk(cudaMallocHost(&b->h_best, std::max<int64_t>(1, b->best_bytes)), "cudaMallocHost best");
    chk(cudaMallocHost(&b->h_bestfit, sizeof(double) * n), "cudaMallocHost best fit");
    chk(cudaMalloc(&b->d_counters, sizeof(int) * std::max<size_t>(1, b->groups.size())),
        "cudaMalloc counters");
    chk(cudaMalloc(&b->d_stamp, sizeof(unsigned long long) * (n + 1)), "cudaMalloc stamps");
    chk(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  }
  if (st == PA_OK) {
    const size_t sb = pa::seed_args_bytes();
    std::vector<unsigned char> h(sb * n);
    b->seed_C = pa::seed_batch_cluster(n);
    for (int i = 0; i < n; ++i)
      b->seed_smem =
          std::max(b->seed_smem, pa::seed_fill_args(b->ctx[i], h.data() + sb * i, b->seed_C));
    if (chk(cudaMalloc(&b->d_seed_args, h.size()), "cudaMalloc seed args"))
      chk(cudaMemcpy(b->d_seed_args, h.data(), h.size(), cudaMemcpyHostToDevice), "copy seed args");
    // one seeding pass now: prepares the kernel outside any later capture
    if (st == PA_OK)
      chk(pa::launch_seed_batch(b->d_seed_args, n, b->seed_smem, b->seed_C, b->stream), "seed");
    if (st == PA_OK) chk(cudaStreamSynchronize(b->stream), "seed sync");
  }
  for (auto& g : b->groups) {
    if (st != PA_OK) break;
    if (!chk(cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking), "stream")) break;
    if (!chk(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming), "event")) break;
    // the default size if it fits, else the nearest larger one, else smaller
    const int C0 = default_cluster(b, g);
    std::vector<int> order{C0};
    for (int C = C0 * 2; C <= 16; C *= 2) order.push_back(C);
    for (int C = C0 / 2; C >= 1; C /= 2) order.push_back(C);
    pa_status gs = PA_EUNSUPPORTED;
    for (int C : order) {
      gs = build_group_args(b, g, C, 1, 1024, false);
      if (gs != PA_EUNSUPPORTED) break;
    }
    if (gs != PA_OK) st = bfail(b, gs, "an instance of the batch does not fit the solve kernel");
  }
  if (st != PA_OK) {
    pa::set_thread_error(b->err);
    destroy_batch(b);
    return st;
  }
  *out = b;
  return PA_OK;
}

void pa_batch_destroy(pa_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  destroy_batch(b);
}

const char* pa_batch_last_error(const pa_batch* b) { return b ? b->err.c_str() : ""; }

pa_status pa_batch_load(pa_batch* b, int32_t i, const double* beta, const int32_t* user_xy_mm,
                        const int32_t* bs_xy_mm) {
  if (!b) return PA_EINVAL;
  if (i < 0 || i >= b->n) return bfail(b, PA_EINVAL, "instance index out of range");
  const bool had = b->ctx[i]->has_positions != 0;
  if ((user_xy_mm != nullptr) != had)
    return bfail(b, PA_EINVAL, "positions must be given exactly when the instance had them");
  pa_status st = pa_load_instance(b->ctx[i], beta, user_xy_mm, bs_xy_mm);
  if (st != PA_OK) return bfail(b, st, pa_last_error(b->ctx[i]));
  return PA_OK;
}

pa_status pa_batch_tune(pa_batch* b, int32_t generations, int32_t* chosen) {
  if (!b) return PA_EINVAL;
  if (generations < 1) return bfail(b, PA_EINVAL, "generations must be >= 1");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pa_status st = bcuda(b, cudaEventCreate(&e0), "event");
  if (st == PA_OK) st = bcuda(b, cudaEventCreate(&e1), "event");
  // The groups run concurrently, so a shape is judged by the whole batch's
  // time: coordinate descent over the groups, each trying every shape that
  // fits while the others keep theirs (seeding included, the same in every
  // run).  Second of two runs counts.
  auto time_all = [&](float* ms) {
    for (int rep = 0; rep < 2 && st == PA_OK; ++rep) {
      cudaEventRecord(e0, b->stream);
      st = run_groups(b, b->stream);
      if (st != PA_OK) break;
      cudaEventRecord(e1, b->stream);
      st = bcuda(b, cudaEventSynchronize(e1), "tune sync");
      if (st == PA_OK) cudaEventElapsedTime(ms, e0, e1);
    }
  };
  for (auto& g : b->groups)
    if (st == PA_OK) st = build_group_args(b, g, g.C, generations, g.threads, g.latency);
  for (size_t k = 0; k < b->groups.size() && st == PA_OK; ++k) {
    auto& g = b->groups[k];
    int best_C = g.C, best_T = g.threads;
    bool best_lat = g.latency;
    float best_ms = 0.f;
    time_all(&best_ms);
    // the tiling choice: clusters of 1024-thread CTAs (one CTA per SM; the
    // throughput column split, or the one-instance latency split) or of
    // 256-thread CTAs (four per SM, several instances sharing an SM), each
    // with 1 to 16 CTAs per instance
    struct Tiling {
      int T;
      bool lat;
    };
    for (const Tiling tl : {Tiling{1024, false}, Tiling{1024, true}, Tiling{256, false}})
      for (int C : {1, 2, 4, 8, 16}) {
        const int T = tl.T;
        if (st != PA_OK) break;
        if (T == best_T && tl.lat == best_lat && C == best_C) continue;
        pa_status gs = build_group_args(b, g, C, generations, T, tl.lat);
        if (gs == PA_EUNSUPPORTED) continue;
        if (gs != PA_OK) {
          st = gs;
          break;
        }
        float ms = 0.f;
        time_all(&ms);
        if (st == PA_OK && ms < best_ms) {
          best_ms = ms;
          best_C = C;
          best_T = T;
          best_lat = tl.lat;
        }
      }
    if (st == PA_OK) st = build_group_args(b, g, best_C, generations, best_T, best_lat);
    // then how much of the GPU the group's persistent clusters may hold at
    // once: all that fits, or less, leaving SMs to the groups running beside
    int best_cap = g.cap8;
    for (int cap8 : {8, 7, 6, 5, 4}) {
      if (st != PA_OK || cap8 == best_cap) continue;
      g.cap8 = cap8;
      st = build_group_args(b, g, best_C, generations, best_T, best_lat);
      if (st != PA_OK) break;
      float ms = 0.f;
      time_all(&ms);
      if (st == PA_OK && ms < best_ms) {
        best_ms = ms;
        best_cap = cap8;
      }
    }
    g.cap8 = best_cap;
    if (st == PA_OK) st = build_group_args(b, g, best_C, generations, best_T, best_lat);
    if (chosen && st == PA_OK) chosen[k] = best_C;
  }
  for (auto& g : b->groups)  // arguments of one generation until the next solve rebuilds them
    if (st == PA_OK) st = build_group_args(b, g, g.C, 1, g.threads, g.latency);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->graph_G = -1;  // the captured graph used the previous shapes
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return st;
}

pa_status pa_batch_groups(pa_batch* b, int32_t* n_groups, int32_t* cluster_sizes,
                          int32_t* cta_threads, int32_t* latency_split,
                          int32_t* resident_clusters, int32_t* group_of_instance) {
  if (!b) return PA_EINVAL;
  if (n_groups) *n_groups = (int32_t)b->groups.size();
  for (size_t k = 0; k < b->groups.size(); ++k) {
    if (cluster_sizes) cluster_sizes[k] = b->groups[k].C;
    if (cta_threads) cta_threads[k] = b->groups[k].threads;
    if (latency_split) latency_split[k] = b->groups[k].latency ? 1 : 0;
    if (resident_clusters) resident_clusters[k] = b->groups[k].clusters;
    if (group_of_instance)
      for (int i : b->groups[k].members) group_of_instance[i] = (int32_t)k;
  }
  return PA_OK;
}

pa_status pa_batch_solve(pa_batch* b, int32_t generations, uint8_t* best_host, double* best_fit) {
  if (!b) return PA_EINVAL;
  if (generations < 0) return bfail(b, PA_EINVAL, "generations must be >= 0");
  pa_status st = PA_OK;
  if (b->graph_G != generations || !b->graph) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    for (auto& g : b->groups) {
      st = build_group_args(b, g, g.C, generations, g.threads, g.latency);
      if (st != PA_OK) return bfail(b, st, "rebuilding batch arguments failed");
    }
    cudaGraph_t graph = nullptr;
    st = bcuda(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
               "begin capture");
    if (st != PA_OK) return st;
    pa_status rs = run_groups(b, b->stream);
    if (rs == PA_OK)
      rs = bcuda(b, cudaMemcpyAsync(b->h_best, b->d_best, std::max<int64_t>(1, b->best_bytes),
                                    cudaMemcpyDeviceToHost, b->stream),
                 "copy best");
    if (rs == PA_OK)
      rs = bcuda(b, cudaMemcpyAsync(b->h_bestfit, b->d_bestfit, sizeof(double) * b->n,
                                    cudaMemcpyDeviceToHost, b->stream),
                 "copy best fit");
    cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
    if (rs != PA_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rs;
    }
    st = bcuda(b, ee, "end capture");
    if (st == PA_OK) st = bcuda(b, cudaGraphInstantiate(&b->graph, graph, 0), "instantiate graph");
    if (graph) cudaGraphDestroy(graph);
    if (st != PA_OK) return st;
    b->graph_G = generations;
  }
  st = bcuda(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
  if (st == PA_OK) st = bcuda(b, cudaStreamSynchronize(b->stream), "sync");
  if (st != PA_OK) return st;
  for (pa_ctx* c : b->ctx) {
    c->cur = 1;
    c->generation = generations;
  }
  if (best_host) std::memcpy(best_host, b->h_best, (size_t)b->best_bytes);
  if (best_fit) std::memcpy(best_fit, b->h_bestfit, sizeof(double) * b->n);
  return PA_OK;
}

pa_status pa_batch_completion_times(pa_batch* b, double* ms_host) {
  if (!b || !ms_host) return PA_EINVAL;
  std::vector<unsigned long long> t(b->n + 1);
  pa_status st = bcuda(b, cudaMemcpyAsync(t.data(), b->d_stamp, sizeof(t[0]) * t.size(),
                                          cudaMemcpyDeviceToHost, b->stream),
                       "copy stamps");
  if (st == PA_OK) st = bcuda(b, cudaStreamSynchronize(b->stream), "sync");
  if (st != PA_OK) return st;
  for (int i = 0; i < b->n; ++i) ms_host[i] = (double)(long long)(t[i] - t[b->n]) * 1e-6;
  return PA_OK;
}

pa_status pa_batch_context(pa_batch* b, int32_t i, pa_ctx** out) {
  if (!b || !out || i < 0 || i >= b->n) return PA_EINVAL;
  *out = b->ctx[i];
  return PA_OK;
}

}  // extern "C"
