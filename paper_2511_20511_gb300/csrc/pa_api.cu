// pa_api.cu -- the C ABI declared in include/pa.h: argument validation,
// context lifetime, device memory, and the host-side sequencing of the
// kernels (every step of the method runs in the kernels of pa_prep.cu,
// pa_fitness.cu and pa_ga.cu).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pa_internal.cuh"

#include <atomic>

namespace pa {

static std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_create_error;  // last pa_create failure of this thread
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void f32_geometry(int L, int K, int* NJ, int* RS, int* vec);

pa_status fail(pa_ctx* ctx, pa_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

pa_status cuda_check(pa_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PA_OK;
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  if (ctx) ctx->err = buf;
  return e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA;
}

}  // namespace pa

using pa::cuda_check;
using pa::fail;

#define PA_TRY(ctx, expr, what)                                \
  do {                                                         \
    pa_status _s = cuda_check((ctx), (expr), (what));          \
    if (_s != PA_OK) return _s;                                \
  } while (0)

namespace pa {
bool instance_ok(const pa_config& c, const double* beta, const int32_t* user_xy_mm,
                 const int32_t* bs_xy_mm, double* bmax) {
  const int64_t n_beta = (int64_t)c.L * c.L * c.K;
  double m = 0.0;
  for (int64_t i = 0; i < n_beta; ++i) {
    const double b = beta[i];
    if (!(b > 0.0) || !std::isfinite(b)) return false;
    m = b > m ? b : m;
  }
  *bmax = m;
  if (user_xy_mm) {
    for (int l = 0; l < c.L; ++l)
      for (int k = 0; k < c.K; ++k) {
        const int64_t u = (int64_t)l * c.K + k;
        const int64_t fx = (int64_t)user_xy_mm[2 * u] - bs_xy_mm[2 * l];
        const int64_t fy = (int64_t)user_xy_mm[2 * u + 1] - bs_xy_mm[2 * l + 1];
        if (fx > INT32_MAX || fx < INT32_MIN || fy > INT32_MAX || fy < INT32_MIN) return false;
      }
  }
  return true;
}
}  // namespace pa

// Copy one instance (beta, positions) into a context's device buffers and
// rebuild its fitness tables.  Buffers must already exist.
static pa_status upload_instance(pa_ctx* c, const double* beta, const int32_t* user_xy_mm,
                                 const int32_t* bs_xy_mm, double bmax) {
  const pa_config& cfg = c->cfg;
  const int L = cfg.L, K = cfg.K;
  const int64_t n_beta = (int64_t)L * L * K, LK = (int64_t)L * K;
  PA_TRY(c, cudaMemcpyAsync(c->beta64, beta, sizeof(double) * n_beta, cudaMemcpyHostToDevice,
                            c->stream),
         "copy beta");
  if (cfg.prec == PA_FP32) {
    int e2 = 0;
    std::frexp(bmax, &e2);  // bmax = f 2^e2, f in [0.5, 1): scaled gains lie in (0, 1)
    c->t32.scale_exp = -e2;
    c->t32.scale = std::ldexp(1.0, -e2);
    c->t32.M = (float)cfg.M;
    c->t32.pc = (float)std::ldexp(c->pc, -e2);
  }
  if (user_xy_mm) {
    PA_TRY(c, cudaMemcpyAsync(c->user_xy, user_xy_mm, sizeof(int32_t) * 2 * LK,
                              cudaMemcpyHostToDevice, c->stream),
           "copy user positions");
    PA_TRY(c, cudaMemcpyAsync(c->bs_xy, bs_xy_mm, sizeof(int32_t) * 2 * L, cudaMemcpyHostToDevice,
                              c->stream),
           "copy BS positions");
  }
  c->has_positions = user_xy_mm != nullptr;
  PA_TRY(c, pa::launch_prep(c), "prepare tables");
  return PA_OK;
}

extern "C" {

const char* pa_status_str(pa_status s) {
  switch (s) {
    case PA_OK: return "ok";
    case PA_EINVAL: return "invalid argument";
    case PA_ENOMEM: return "out of memory";
    case PA_ECUDA: return "CUDA error";
    case PA_ETIMEOUT: return "device wait timed out";
    case PA_EUNSUPPORTED: return "unsupported configuration";
    case PA_EBUSY: return "busy";
  }
  return "unknown status";
}

const char* pa_last_error(const pa_ctx* ctx) {
  return ctx ? ctx->err.c_str() : pa::t_create_error.c_str();
}

uint64_t pa_kernel_launches(void) { return pa::g_launches.load(std::memory_order_relaxed); }

pa_status pa_solve_cluster_ctas(const pa_ctx* ctx, int32_t* ctas) {
  if (!ctx || !ctas) return PA_EINVAL;
  *ctas = ctx->t32.streamed ? 0 : ctx->solve_C;
  return PA_OK;
}

uint64_t pa_prob_to_thresh(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return 1ULL << 32;
  return (uint64_t)std::floor(p * 4294967296.0);
}

pa_status pa_config_default(pa_config* c, int32_t L, int32_t K) {
  if (!c) return PA_EINVAL;
  std::memset(c, 0, sizeof *c);
  c->L = L;
  c->K = K;
  c->tau_p = K;
  c->mode = PA_SINR_ASYMPTOTIC;
  c->M = 256.0;
  c->rho = 10.0 / std::pow(500.0, -3.8);
  c->sigma2 = 1.0;
  c->prec = PA_FP32;
  c->N = 256;
  c->E = 2;
  c->tour = 3;
  c->pc_thresh = pa_prob_to_thresh(0.9);
  c->pm_thresh = pa_prob_to_thresh(0.05);
  c->seed = 0;
  c->kmeans_k = K;
  c->kmeans_max_iter = 100;
  c->n_seeded = (c->N + 1) / 2;
  c->objective = PA_OBJ_SUM_SE;
  c->islands = 0;
  c->recluster = 3;
  c->island_iter = 100;
  return PA_OK;
}

static pa_status validate_config(const pa_config* c, std::string* why) {
  auto bad = [&](const char* m) {
    *why = m;
    return PA_EINVAL;
  };
  if (c->L < 2 || c->L > pa::kMaxL) return bad("L must be in [2, 255]");
  if (c->K < 1 || c->K > pa::kMaxK) return bad("K must be in [1, 64]");
  if ((int64_t)c->L * c->K > 64 * 64) return bad("L*K must be <= 4096");
  if (c->mode != PA_SINR_ASYMPTOTIC && c->mode != PA_SINR_FINITE_M) return bad("unknown mode");
  if (c->prec != PA_FP32 && c->prec != PA_FP64) return bad("unknown precision");
  if (c->mode == PA_SINR_FINITE_M) {
    if (c->tau_p < 1) return bad("tau_p must be >= 1");
    if (!(c->M > 0.0) || !std::isfinite(c->M)) return bad("M must be finite and > 0");
    if (!(c->rho > 0.0) || !std::isfinite(c->rho)) return bad("rho must be finite and > 0");
    if (!(c->sigma2 >= 0.0) || !std::isfinite(c->sigma2)) return bad("sigma2 must be >= 0");
  }
  if (c->N < 2 || c->N > (1 << 24)) return bad("N must be in [2, 2^24]");
  if (c->E < 0 || c->E >= c->N || c->E > 64) return bad("E must be in [0, min(N-1, 64)]");
  if (c->tour < 1 || c->tour > 64) return bad("tour must be in [1, 64]");
  if (c->pc_thresh > (1ULL << 32) || c->pm_thresh > (1ULL << 32))
    return bad("thresholds must be <= 2^32");
  if (c->kmeans_k < 1 || c->kmeans_k > c->K) return bad("kmeans_k must be in [1, K]");
  if (c->kmeans_max_iter < 1) return bad("kmeans_max_iter must be >= 1");
  if (c->n_seeded < 0 || c->n_seeded > c->N) return bad("n_seeded must be in [0, N]");
  if ((c->flags & ~PA_FLAG_TEST_STALL_COPIES) != 0) return bad("unknown flags");
  if (c->objective != PA_OBJ_SUM_SE && c->objective != PA_OBJ_MIN_SINR)
    return bad("unknown objective");
  if (c->islands < 0 || c->islands > pa::kMaxIslands) return bad("islands must be in [0, 64]");
  if (c->recluster < 0 || c->island_iter < 0) return bad("recluster and island_iter must be >= 0");
  if (c->islands >= 2) {
    if (c->N > pa::kMaxIslandN) return bad("islands need N <= 4096");
    if (c->islands > c->N) return bad("islands must be <= N");
    if (c->recluster < 1 || c->island_iter < 1)
      return bad("islands need recluster >= 1 and island_iter >= 1");
  }
  for (int i = 0; i < 2; ++i)
    if (c->reserved[i] != 0) return bad("reserved fields must be 0");
  return PA_OK;
}

static void free_ctx(pa_ctx* c) {
  if (!c) return;
  cudaFree(c->arena);
  cudaFree(c->t32.partial);
  cudaFreeHost(c->h_best);
  cudaFree(c->stage_pop);
  cudaFree(c->stage_fit);
  delete c;
}

// Device bytes of the best-member slot: the row, then its FP64 fitness at
// the next 8-byte boundary.
static size_t best_bytes(int64_t LK) { return (size_t)(((LK + 7) & ~int64_t(7)) + 8); }

pa_status pa_create(const pa_config* cfg, const double* beta, const int32_t* user_xy_mm,
                    const int32_t* bs_xy_mm, void* stream, pa_ctx** out) {
  std::string& why = pa::t_create_error;
  why.clear();
  auto reject = [&](pa_status s, const char* m) {
    why = m;
    return s;
  };
  if (!out) return reject(PA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || !beta) return reject(PA_EINVAL, "cfg and beta are required");
  if ((user_xy_mm == nullptr) != (bs_xy_mm == nullptr))
    return reject(PA_EINVAL, "user and BS positions must both be given or both be NULL");
  if (validate_config(cfg, &why) != PA_OK) return PA_EINVAL;
  double bmax = 0.0;
  if (!pa::instance_ok(*cfg, beta, user_xy_mm, bs_xy_mm, &bmax))
    return reject(PA_EINVAL, "beta must be finite and > 0; relative positions within int32");
  const int L = cfg->L, K = cfg->K;
  int sJT = 0, sRSt = 0, svec = 0, sntile = 0;
  const bool resident = cfg->prec != PA_FP32 || pa::f32_supported(L, K, nullptr);
  if (!resident && !pa::f32_stream_geometry(L, K, &sJT, &sRSt, &svec, &sntile))
    return reject(PA_EUNSUPPORTED, "FP32 gain table of this (L, K) exceeds shared memory");

  pa_ctx* c = new (std::nothrow) pa_ctx();
  if (!c) return PA_ENOMEM;
  c->cfg = *cfg;
  c->test_stall = (cfg->flags & PA_FLAG_TEST_STALL_COPIES) ? 1 : 0;
  c->stream = static_cast<cudaStream_t>(stream);
  c->nc = cfg->sigma2 / cfg->rho;
  c->pc = cfg->sigma2 / ((double)cfg->tau_p * cfg->rho);
  pa_status st = PA_OK;
  auto chk = [&](cudaError_t e, const char* what) {
    if (st == PA_OK) st = cuda_check(c, e, what);
    return st == PA_OK;
  };
  const int64_t n_beta = (int64_t)L * L * K, LK = (int64_t)L * K;
  const size_t fsz = cfg->prec == PA_FP64 ? 8 : 4;
  do {
    if (!chk(cudaGetDevice(&c->device), "cudaGetDevice")) break;
    if (!chk(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device),
             "cudaDeviceGetAttribute"))
      break;
    // every device buffer of the context is carved from one allocation
    // (256-byte aligned parts): creating a context costs one cudaMalloc
    std::vector<std::pair<void**, size_t>> parts;
    auto want = [&](auto** p, size_t bytes) { parts.emplace_back((void**)p, bytes); };
    want(&c->beta64, sizeof(double) * n_beta);
    want(&c->bnc64, sizeof(double) * L);
    if (cfg->prec == PA_FP32 && !resident) {
      c->t32.streamed = 1;
      c->t32.JT = sJT;
      c->t32.RSt = sRSt;
      c->t32.vec = svec;
      c->t32.ntile = sntile;
      c->t32.tile_floats = ((LK * sRSt + 3) / 4) * 4;
      want(&c->t32.tab, sizeof(float) * c->t32.tile_floats * sntile);
    } else if (cfg->prec == PA_FP32) {
      int NJ, RS, vec;
      pa::f32_geometry(L, K, &NJ, &RS, &vec);
      c->t32.NJ = NJ;
      c->t32.RS = RS;
      c->t32.vec = vec;
      want(&c->t32.tab, sizeof(float) * (((LK * RS + 3) / 4) * 4));
    }
    if (cfg->prec == PA_FP32) {
      want(&c->t32.own, sizeof(float) * LK);
      want(&c->t32.bn, sizeof(float) * L);
      want(&c->t32.err_flag, sizeof(int));
    }
    want(&c->user_xy, sizeof(int32_t) * 2 * LK);
    want(&c->bs_xy, sizeof(int32_t) * 2 * L);
    want(&c->labels, sizeof(int32_t) * LK);
    want(&c->centroids, sizeof(double) * 2 * cfg->kmeans_k);
    want(&c->pop[0], (size_t)cfg->N * LK);
    want(&c->pop[1], (size_t)cfg->N * LK);
    want(&c->fit, fsz * cfg->N);
    want(&c->scratch_i64, sizeof(int64_t) * 8);
    // best row, then its fitness at the next 8-byte boundary (one copy back)
    want(&c->best_row, best_bytes(LK));
    if (cfg->islands >= 2) {
      const size_t n4 = sizeof(int32_t) * cfg->N;
      want(&c->isl_label, n4);
      for (pa::IslandLists* il : {&c->isl_res, &c->isl_usr}) {
        want(&il->list, n4);
        want(&il->pos, n4);
        want(&il->off, sizeof(int32_t) * (cfg->islands + 1));
      }
      want(&c->isl_passes, sizeof(int32_t));
      if (!pa::island_cnt_in_smem(cfg->N, L, K, cfg->islands))
        want(&c->isl_cnt, sizeof(uint32_t) * pa::island_cnt_words(L, K, cfg->islands));
    }
    size_t total = 0;
    for (auto& pt : parts) total = ((total + 255) & ~size_t(255)) + pt.second;
    if (!chk(cudaMalloc(&c->arena, total), "cudaMalloc context")) break;
    size_t off = 0;
    for (auto& pt : parts) {
      off = (off + 255) & ~size_t(255);
      *pt.first = static_cast<unsigned char*>(c->arena) + off;
      off += pt.second;
    }
    if (cfg->prec == PA_FP32 &&
        !chk(cudaMemsetAsync(c->t32.err_flag, 0, sizeof(int), c->stream), "memset flag"))
      break;
    if (cfg->islands >= 2 &&
        !chk(cudaMemsetAsync(c->isl_label, 0xFF, sizeof(int32_t) * cfg->N, c->stream),
             "memset islands"))
      break;
    st = upload_instance(c, beta, user_xy_mm, bs_xy_mm, bmax);
    if (st != PA_OK) break;
    if (!chk(cudaStreamSynchronize(c->stream), "prepare sync")) break;
  } while (0);
  if (st != PA_OK) {
    why = c->err;
    free_ctx(c);
    return st;
  }
  *out = c;
  return PA_OK;
}

pa_status pa_load_instance(pa_ctx* ctx, const double* beta, const int32_t* user_xy_mm,
                           const int32_t* bs_xy_mm) {
  if (!ctx) return PA_EINVAL;
  if (!beta) return fail(ctx, PA_EINVAL, "null beta");
  if ((user_xy_mm == nullptr) != (bs_xy_mm == nullptr))
    return fail(ctx, PA_EINVAL, "user and BS positions must both be given or both be NULL");
  double bmax = 0.0;
  if (!pa::instance_ok(ctx->cfg, beta, user_xy_mm, bs_xy_mm, &bmax))
    return fail(ctx, PA_EINVAL, "beta must be finite and > 0; positions within int32");
  pa_status st = upload_instance(ctx, beta, user_xy_mm, bs_xy_mm, bmax);
  if (st != PA_OK) return st;
  ctx->cur = 0;
  ctx->generation = 0;
  ctx->isl_valid = 0;
  return PA_OK;
}

void pa_destroy(pa_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

pa_status pa_set_seed(pa_ctx* ctx, uint64_t seed) {
  if (!ctx) return PA_EINVAL;
  ctx->cfg.seed = seed;
  return PA_OK;
}

pa_status pa_set_stream(pa_ctx* ctx, void* stream) {
  if (!ctx) return PA_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return PA_OK;
}

static cudaError_t eval_any(pa_ctx* ctx, const uint8_t* pop, int64_t n, void* fit) {
  if (ctx->cfg.prec == PA_FP64)
    return pa::launch_eval_f64(ctx, pop, n, static_cast<double*>(fit), ctx->stream);
  ctx->wait_check = 1;
  if (ctx->t32.streamed)
    return pa::launch_eval_f32_stream(ctx, pop, n, static_cast<float*>(fit), ctx->stream);
  return pa::launch_eval_f32(ctx, pop, n, static_cast<float*>(fit), ctx->stream);
}

// A bounded device wait of an earlier kernel that gave up (shared-memory
// staging of the FP32 evaluations): reported once, then cleared.
static pa_status check_timeout(pa_ctx* ctx) {
  if (!ctx->t32.err_flag || !ctx->wait_check) return PA_OK;
  ctx->wait_check = 0;
  int flag = 0;
  PA_TRY(ctx, cudaMemcpy(&flag, ctx->t32.err_flag, sizeof flag, cudaMemcpyDeviceToHost),
         "read flag");
  if (!flag) return PA_OK;
  cudaMemset(ctx->t32.err_flag, 0, sizeof(int));
  return fail(ctx, PA_ETIMEOUT, "a shared-memory tile copy did not complete in time");
}

pa_status pa_eval_population(pa_ctx* ctx, const uint8_t* pop_dev, int64_t n, void* fit_dev) {
  if (!ctx) return PA_EINVAL;
  if (n < 0) return fail(ctx, PA_EINVAL, "n must be >= 0");
  if (n == 0) return PA_OK;
  if (!pop_dev || !fit_dev) return fail(ctx, PA_EINVAL, "null buffer");
  PA_TRY(ctx, eval_any(ctx, pop_dev, n, fit_dev), "eval kernel");
  return PA_OK;
}

static pa_status ensure_stage(pa_ctx* ctx, int64_t n) {
  if (n <= ctx->stage_cap) return PA_OK;
  cudaFree(ctx->stage_pop);
  cudaFree(ctx->stage_fit);
  ctx->stage_pop = nullptr;
  ctx->stage_fit = nullptr;
  ctx->stage_cap = 0;
  const int64_t LK = (int64_t)ctx->cfg.L * ctx->cfg.K;
  const size_t fsz = ctx->cfg.prec == PA_FP64 ? 8 : 4;
  PA_TRY(ctx, cudaMalloc(&ctx->stage_pop, (size_t)(n * LK)), "cudaMalloc staging");
  PA_TRY(ctx, cudaMalloc(&ctx->stage_fit, fsz * (size_t)n), "cudaMalloc staging");
  ctx->stage_cap = n;
  return PA_OK;
}

pa_status pa_eval_population_host(pa_ctx* ctx, const uint8_t* pop_host, int64_t n,
                                  void* fit_host) {
  if (!ctx) return PA_EINVAL;
  if (n < 0) return fail(ctx, PA_EINVAL, "n must be >= 0");
  if (n == 0) return PA_OK;
  if (!pop_host || !fit_host) return fail(ctx, PA_EINVAL, "null buffer");
  pa_status st = ensure_stage(ctx, n);
  if (st != PA_OK) return st;
  const int64_t LK = (int64_t)ctx->cfg.L * ctx->cfg.K;
  const size_t fsz = ctx->cfg.prec == PA_FP64 ? 8 : 4;
  PA_TRY(ctx, cudaMemcpyAsync(ctx->stage_pop, pop_host, (size_t)(n * LK), cudaMemcpyHostToDevice,
                              ctx->stream),
         "copy population");
  PA_TRY(ctx, eval_any(ctx, ctx->stage_pop, n, ctx->stage_fit), "eval kernel");
  PA_TRY(ctx, cudaMemcpyAsync(fit_host, ctx->stage_fit, fsz * (size_t)n, cudaMemcpyDeviceToHost,
                              ctx->stream),
         "copy fitness");
  PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  return check_timeout(ctx);
}

pa_status pa_ga_step(pa_ctx* ctx, const uint8_t* pop_dev, const void* fit_dev, int32_t generation,
                     uint8_t* next_dev) {
  if (!ctx) return PA_EINVAL;
  if (!pop_dev || !fit_dev || !next_dev) return fail(ctx, PA_EINVAL, "null buffer");
  if (generation < 0) return fail(ctx, PA_EINVAL, "generation must be >= 0");
  const size_t bytes = (size_t)ctx->cfg.N * ctx->cfg.L * ctx->cfg.K;
  const uint8_t* a0 = pop_dev;
  const uint8_t* b0 = next_dev;
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(ctx, PA_EINVAL, "buffers overlap");
  PA_TRY(ctx, pa::launch_ga_step(ctx, pop_dev, fit_dev, generation, next_dev, ctx->stream),
         "ga kernel");
  return PA_OK;
}

pa_status pa_kmeans_seed(pa_ctx* ctx, int32_t* labels_host, double* centroids_host) {
  if (!ctx) return PA_EINVAL;
  if ((labels_host || centroids_host) && !ctx->has_positions)
    return fail(ctx, PA_EINVAL, "no positions: K-means outputs unavailable");
  ctx->cur = 0;
  ctx->generation = 0;
  ctx->isl_valid = 0;
  PA_TRY(ctx, pa::launch_seed(ctx, ctx->pop[0], ctx->stream), "seed kernel");
  const int64_t LK = (int64_t)ctx->cfg.L * ctx->cfg.K;
  if (labels_host)
    PA_TRY(ctx, cudaMemcpyAsync(labels_host, ctx->labels, sizeof(int32_t) * LK,
                                cudaMemcpyDeviceToHost, ctx->stream),
           "copy labels");
  if (centroids_host)
    PA_TRY(ctx, cudaMemcpyAsync(centroids_host, ctx->centroids,
                                sizeof(double) * 2 * ctx->cfg.kmeans_k, cudaMemcpyDeviceToHost,
                                ctx->stream),
           "copy centroids");
  if (labels_host || centroids_host) PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  return PA_OK;
}

// G generations on the resident population.  One fused cluster launch
// (pa_solve.cu) when the instance fits; otherwise one evaluation and one GA
// launch per generation.  Either way the fitness buffer ends up holding the
// fitness of the population it left behind only in the fused case.
static pa_status run_generations(pa_ctx* ctx, int32_t generations, bool* final_evaluated) {
  *final_evaluated = false;
  if (generations == 0) return PA_OK;
  if (ctx->cfg.islands >= 2) {
    // Alg. 2: every `recluster` generations (and whenever the labels do not
    // belong to this population) K-means into islands and their member
    // lists, and island generations in between.  All of it in one cluster
    // launch of the fused solve in island mode, the K-means included, where
    // that fits in shared memory; else per block of generations up to the
    // next re-clustering: the K-means and list kernels, then one fused
    // launch (or, where that does not fit either, one generation at a time:
    // fitness, one island generation).  The fused launches leave the final
    // population's fitness.
    {
      const cudaError_t e = pa::launch_solve(ctx, ctx->pop[ctx->cur], ctx->pop[ctx->cur ^ 1],
                                             ctx->generation, generations, ctx->fit, nullptr,
                                             nullptr, ctx->stream, ctx->isl_label,
                                             &ctx->isl_res, true);
      if (e == cudaSuccess) {
        ctx->cur ^= 1;
        ctx->generation += generations;
        ctx->isl_valid = 1;
        *final_evaluated = true;
        return PA_OK;
      }
      if (e != cudaErrorNotSupported) return cuda_check(ctx, e, "island solve kernel");
    }
    int32_t done = 0;
    while (done < generations) {
      uint8_t* cur = ctx->pop[ctx->cur];
      uint8_t* nxt = ctx->pop[ctx->cur ^ 1];
      const int R = ctx->cfg.recluster;
      if (!ctx->isl_valid || ctx->generation % R == 0) {
        PA_TRY(ctx, pa::launch_island_kmeans(ctx, cur, ctx->generation, ctx->isl_label,
                                             ctx->stream),
               "island K-means kernel");
        PA_TRY(ctx, pa::launch_island_lists(ctx, ctx->isl_label, ctx->isl_res, ctx->stream),
               "island lists kernel");
        ctx->isl_valid = 1;
      }
      const int32_t block = std::min(generations - done, R - ctx->generation % R);
      const cudaError_t e = pa::launch_solve(ctx, cur, nxt, ctx->generation, block, ctx->fit,
                                             nullptr, nullptr, ctx->stream, ctx->isl_label,
                                             &ctx->isl_res);
      if (e == cudaSuccess) {
        ctx->cur ^= 1;
        ctx->generation += block;
        done += block;
        *final_evaluated = true;
        continue;
      }
      if (e != cudaErrorNotSupported) return cuda_check(ctx, e, "island solve kernel");
      PA_TRY(ctx, eval_any(ctx, cur, ctx->cfg.N, ctx->fit), "eval kernel");
      PA_TRY(ctx, pa::launch_island_step(ctx, cur, ctx->fit, ctx->isl_label, ctx->isl_res,
                                         ctx->generation, nxt, ctx->stream),
             "island step kernel");
      ctx->cur ^= 1;
      ctx->generation += 1;
      done += 1;
      *final_evaluated = false;
    }
    return PA_OK;
  }
  {
    cudaError_t e = pa::launch_solve(ctx, ctx->pop[ctx->cur], ctx->pop[ctx->cur ^ 1],
                                     ctx->generation, generations, ctx->fit, nullptr, nullptr,
                                     ctx->stream);
    if (e == cudaSuccess) {
      ctx->cur ^= 1;
      ctx->generation += generations;
      *final_evaluated = true;
      return PA_OK;
    }
    if (e != cudaErrorNotSupported) return cuda_check(ctx, e, "solve kernel");
  }
  for (int32_t g = 0; g < generations; ++g) {
    uint8_t* cur = ctx->pop[ctx->cur];
    uint8_t* nxt = ctx->pop[ctx->cur ^ 1];
    PA_TRY(ctx, eval_any(ctx, cur, ctx->cfg.N, ctx->fit), "eval kernel");
    PA_TRY(ctx, pa::launch_ga_step(ctx, cur, ctx->fit, ctx->generation, nxt, ctx->stream),
           "ga kernel");
    ctx->cur ^= 1;
    ctx->generation += 1;
  }
  return PA_OK;
}

pa_status pa_step(pa_ctx* ctx, int32_t generations) {
  if (!ctx) return PA_EINVAL;
  if (generations < 0) return fail(ctx, PA_EINVAL, "generations must be >= 0");
  bool evaluated = false;
  return run_generations(ctx, generations, &evaluated);
}

pa_status pa_solve(pa_ctx* ctx, int32_t generations, uint8_t* best_host, double* best_fit) {
  if (!ctx) return PA_EINVAL;
  if (generations < 0) return fail(ctx, PA_EINVAL, "generations must be >= 0");
  pa_status st = pa_kmeans_seed(ctx, nullptr, nullptr);
  if (st != PA_OK) return st;
  const int64_t LK = (int64_t)ctx->cfg.L * ctx->cfg.K;
  double* best_dev = reinterpret_cast<double*>(ctx->best_row + ((LK + 7) & ~int64_t(7)));
  // fused path: all generations, the final evaluation and the best member
  // in one cluster launch (Alg. 1 only; islands launch once per
  // re-clustering)
  cudaError_t e = ctx->cfg.islands >= 2
                      ? cudaErrorNotSupported
                      : pa::launch_solve(ctx, ctx->pop[0], ctx->pop[1], 0, generations, ctx->fit,
                                         ctx->best_row, best_dev, ctx->stream);
  if (e == cudaSuccess) {
    ctx->cur = 1;
    ctx->generation = generations;
  } else if (e == cudaErrorNotSupported) {
    bool evaluated = false;
    st = run_generations(ctx, generations, &evaluated);
    if (st != PA_OK) return st;
    uint8_t* cur = ctx->pop[ctx->cur];
    if (!evaluated) PA_TRY(ctx, eval_any(ctx, cur, ctx->cfg.N, ctx->fit), "eval kernel");
    PA_TRY(ctx, pa::launch_argbest(ctx, ctx->fit, cur, ctx->best_row, best_dev, ctx->stream),
           "argbest kernel");
  } else {
    return cuda_check(ctx, e, "solve kernel");
  }
  // the best row and its fitness come back in one copy to pinned memory
  if ((best_host || best_fit) && !ctx->h_best)
    PA_TRY(ctx, cudaMallocHost(&ctx->h_best, best_bytes(LK)), "cudaMallocHost best");
  if (best_host || best_fit)
    PA_TRY(ctx, cudaMemcpyAsync(ctx->h_best, ctx->best_row, best_bytes(LK),
                                cudaMemcpyDeviceToHost, ctx->stream),
           "copy best");
  PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  if (best_host) std::memcpy(best_host, ctx->h_best, (size_t)LK);
  if (best_fit) std::memcpy(best_fit, ctx->h_best + ((LK + 7) & ~int64_t(7)), sizeof(double));
  return check_timeout(ctx);
}

pa_status pa_get_population(pa_ctx* ctx, uint8_t* pop_host, void* fit_host, int32_t* generation) {
  if (!ctx) return PA_EINVAL;
  const size_t bytes = (size_t)ctx->cfg.N * ctx->cfg.L * ctx->cfg.K;
  uint8_t* cur = ctx->pop[ctx->cur];
  if (pop_host)
    PA_TRY(ctx, cudaMemcpyAsync(pop_host, cur, bytes, cudaMemcpyDeviceToHost, ctx->stream),
           "copy population");
  if (fit_host) {
    PA_TRY(ctx, eval_any(ctx, cur, ctx->cfg.N, ctx->fit), "eval kernel");
    const size_t fsz = ctx->cfg.prec == PA_FP64 ? 8 : 4;
    PA_TRY(ctx, cudaMemcpyAsync(fit_host, ctx->fit, fsz * ctx->cfg.N, cudaMemcpyDeviceToHost,
                                ctx->stream),
           "copy fitness");
  }
  if (generation) *generation = ctx->generation;
  PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  return check_timeout(ctx);
}

pa_status pa_validate_population(pa_ctx* ctx, const uint8_t* pop_dev, int64_t n,
                                 int64_t* first_bad) {
  if (!ctx || !first_bad) return PA_EINVAL;
  if (n < 0) return fail(ctx, PA_EINVAL, "n must be >= 0");
  *first_bad = -1;
  if (n == 0) return PA_OK;
  if (!pop_dev) return fail(ctx, PA_EINVAL, "null buffer");
  int64_t* flag = ctx->scratch_i64 + 1;
  PA_TRY(ctx, cudaMemsetAsync(flag, 0xFF, sizeof(int64_t), ctx->stream), "memset");
  PA_TRY(ctx, pa::launch_validate(ctx, pop_dev, n, flag, ctx->stream), "validate kernel");
  uint64_t h = 0;
  PA_TRY(ctx, cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "copy");
  PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  *first_bad = (h == ~0ULL) ? -1 : (int64_t)h;
  return PA_OK;
}

pa_status pa_set_population(pa_ctx* ctx, const uint8_t* pop_host, int32_t generation) {
  if (!ctx || !pop_host) return PA_EINVAL;
  if (generation < 0) return fail(ctx, PA_EINVAL, "generation must be >= 0");
  const size_t bytes = (size_t)ctx->cfg.N * ctx->cfg.L * ctx->cfg.K;
  uint8_t* dst = ctx->pop[ctx->cur ^ 1];
  PA_TRY(ctx, cudaMemcpyAsync(dst, pop_host, bytes, cudaMemcpyHostToDevice, ctx->stream),
         "copy population");
  int64_t bad = -1;
  pa_status st = pa_validate_population(ctx, dst, ctx->cfg.N, &bad);
  if (st != PA_OK) return st;
  if (bad >= 0) return fail(ctx, PA_EINVAL, "population row is not a permutation");
  ctx->cur ^= 1;
  ctx->generation = generation;
  ctx->isl_valid = 0;
  return PA_OK;
}

pa_status pa_island_cluster(pa_ctx* ctx, const uint8_t* pop_dev, int32_t generation,
                            int32_t* labels_dev, int32_t* passes_host) {
  if (!ctx) return PA_EINVAL;
  if (ctx->cfg.islands < 2) return fail(ctx, PA_EINVAL, "context created without islands");
  if (!pop_dev || !labels_dev) return fail(ctx, PA_EINVAL, "null buffer");
  if (generation < 0) return fail(ctx, PA_EINVAL, "generation must be >= 0");
  PA_TRY(ctx, pa::launch_island_kmeans(ctx, pop_dev, generation, labels_dev, ctx->stream),
         "island K-means kernel");
  if (passes_host) {
    PA_TRY(ctx, cudaMemcpyAsync(passes_host, ctx->isl_passes, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, ctx->stream),
           "copy passes");
    PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  }
  return PA_OK;
}

pa_status pa_island_step(pa_ctx* ctx, const uint8_t* pop_dev, const void* fit_dev,
                         const int32_t* labels_dev, int32_t generation, uint8_t* next_dev) {
  if (!ctx) return PA_EINVAL;
  if (ctx->cfg.islands < 2) return fail(ctx, PA_EINVAL, "context created without islands");
  if (!pop_dev || !fit_dev || !labels_dev || !next_dev) return fail(ctx, PA_EINVAL, "null buffer");
  if (generation < 0) return fail(ctx, PA_EINVAL, "generation must be >= 0");
  const size_t bytes = (size_t)ctx->cfg.N * ctx->cfg.L * ctx->cfg.K;
  const uint8_t* a0 = pop_dev;
  const uint8_t* b0 = next_dev;
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(ctx, PA_EINVAL, "buffers overlap");
  // the caller's labels get member lists of their own: the resident
  // population's islands stay as they are
  PA_TRY(ctx, pa::launch_island_lists(ctx, labels_dev, ctx->isl_usr, ctx->stream),
         "island lists kernel");
  PA_TRY(ctx, pa::launch_island_step(ctx, pop_dev, fit_dev, labels_dev, ctx->isl_usr, generation,
                                     next_dev, ctx->stream),
         "island step kernel");
  return PA_OK;
}

pa_status pa_get_islands(pa_ctx* ctx, int32_t* labels_host) {
  if (!ctx || !labels_host) return PA_EINVAL;
  if (ctx->cfg.islands < 2) return fail(ctx, PA_EINVAL, "context created without islands");
  PA_TRY(ctx, cudaMemcpyAsync(labels_host, ctx->isl_label, sizeof(int32_t) * ctx->cfg.N,
                              cudaMemcpyDeviceToHost, ctx->stream),
         "copy islands");
  PA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  return PA_OK;
}

pa_status pa_population_device(pa_ctx* ctx, uint8_t** pop_dev, void** fit_dev) {
  if (!ctx) return PA_EINVAL;
  if (pop_dev) *pop_dev = ctx->pop[ctx->cur];
  if (fit_dev) *fit_dev = ctx->fit;
  return PA_OK;
}

}  // extern "C"

namespace pa {
// Configuration check and per-thread error text for entry points that run
// without a context.
bool config_ok(const pa_config* c, std::string* why) { return validate_config(c, why) == PA_OK; }
void set_thread_error(const std::string& msg) { t_create_error = msg; }
}  // namespace pa
