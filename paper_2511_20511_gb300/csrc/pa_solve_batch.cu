// pa_solve_batch.cu -- many instances per launch: persistent thread-block
// clusters take the next instance from a counter and run the whole GA on it
// (the same device code as the one-instance kernel, pa_solve_body.cuh); the
// argument records, launch shapes and CTA sizes of the batch and server paths.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "pa_solve_body.cuh"

namespace pa {
namespace {

// Many instances per launch (persistent clusters): each cluster takes the
// next instance index from a global counter until the list is exhausted.
// Instances of one launch share the kernel variant (NJ, VEC, FIN, FT); their
// sizes may differ (shared memory is sized for the largest).
template <typename FT, int NJ, int VEC, bool FIN, int THREADS>
__global__ void __launch_bounds__(THREADS, kSolveThreads / THREADS)
    k_solve_batch(const SolveArgs* __restrict__ insts, int n_inst, int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int elites[64];
  __shared__ int next;
  // the instance's arguments live in shared memory (a local copy would sit
  // in local memory: the kernel runs at the 64-register limit)
  __shared__ SolveArgs sargs;
  static_assert(sizeof(SolveArgs) % 8 == 0, "SolveArgs is copied as 8-byte words");
  constexpr int kArgWords = (int)(sizeof(SolveArgs) / 8);
  static_assert(kArgWords <= THREADS, "one word per thread");
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  for (;;) {
    if (cluster.block_rank() == 0 && threadIdx.x == 0) {
      const int i = atomicAdd(counter, 1);
      for (int r = 0; r < C; ++r) *cluster.map_shared_rank(&next, r) = i;
    }
    cluster.sync();
    const int i = next;
    if (i >= n_inst) break;
    if (threadIdx.x < kArgWords)
      reinterpret_cast<uint64_t*>(&sargs)[threadIdx.x] =
          reinterpret_cast<const uint64_t*>(insts + i)[threadIdx.x];
    __syncthreads();
    solve_body<FT, NJ, VEC, FIN, kBatchMaxNP>(sargs, smem, elites, cluster);
  }
}

}  // namespace

namespace {

template <typename FT, int NJ, int VEC, bool FIN, int THREADS>
cudaError_t run_solve_batch(int C, int clusters, const SolveArgs* d_args, int n, int* d_counter,
                            size_t smem, bool query_only, int* max_clusters, cudaStream_t st) {
  auto kern = k_solve_batch<FT, NJ, VEC, FIN, THREADS>;
  static std::atomic<uint64_t> prepared{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ULL << (dev & 63);
  if (!(prepared.load() & bit)) {
    e = raise_smem_cap((const void*)kern, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    prepared.fetch_or(bit);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * std::max(1, clusters), 1, 1);
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query_only) {
    int m = 0;
    e = cudaOccupancyMaxActiveClusters(&m, kern, &cfg);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      m = 0;
    }
    *max_clusters = m;
    return cudaSuccess;
  }
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  e = cudaLaunchKernelEx(&cfg, kern, d_args, n, d_counter);
  count_launch();
  return e;
}

template <typename FT, int VEC, bool FIN>
cudaError_t pick_batch(int NJ, int C, int clusters, const SolveArgs* d, int n, int* ctr,
                       size_t smem, bool q, int* mc, cudaStream_t st) {
  constexpr int T = kSolveThreads;
  switch (NJ) {
    case 4: return run_solve_batch<FT, 4, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 8: return run_solve_batch<FT, 8, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 12: return run_solve_batch<FT, 12, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 16: return run_solve_batch<FT, 16, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 20: return run_solve_batch<FT, 20, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 24: return run_solve_batch<FT, 24, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 28: return run_solve_batch<FT, 28, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 32: return run_solve_batch<FT, 32, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 36: return run_solve_batch<FT, 36, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 40: return run_solve_batch<FT, 40, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 44: return run_solve_batch<FT, 44, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 48: return run_solve_batch<FT, 48, VEC, FIN, T>(C, clusters, d, n, ctr, smem, q, mc, st);
    default: return cudaErrorInvalidValue;
  }
}


cudaError_t dispatch_batch(const pa_ctx* proto, int C, int clusters, const SolveArgs* d, int n,
                           int* ctr, size_t smem, bool q, int* mc, cudaStream_t st) {
  const pa_config& c = proto->cfg;
  const bool fin = c.mode == PA_SINR_FINITE_M;
  if (c.prec == PA_FP64)
    return run_solve_batch<double, 4, 2, false, kSolveThreads>(C, clusters, d, n, ctr, smem, q,
                                                               mc, st);
  const int NJ = proto->t32.NJ;
  if (proto->t32.vec == 2)
    return fin ? pick_batch<float, 2, true>(NJ, C, clusters, d, n, ctr, smem, q, mc, st)
               : pick_batch<float, 2, false>(NJ, C, clusters, d, n, ctr, smem, q, mc, st);
  return fin ? pick_batch<float, 1, true>(NJ, C, clusters, d, n, ctr, smem, q, mc, st)
             : pick_batch<float, 1, false>(NJ, C, clusters, d, n, ctr, smem, q, mc, st);
}

}  // namespace

size_t solve_args_bytes() { return sizeof(SolveArgs); }

// Arguments of one instance's solve with cluster size C (written to
// args_out, a SolveArgs); returns the shared memory it needs, or 0 when it
// does not fit in one CTA.
size_t solve_fill_args(const pa_ctx* ctx, int C, int gen0, int G, const uint8_t* pop_in,
                       uint8_t* pop_out, void* fit_out, uint8_t* best_row, double* best_fit,
                       void* args_out) {
  const pa_config& c = ctx->cfg;
  if (C > c.N || ctx->t32.streamed) return 0;
  const SolveShape s = solve_shape(ctx, C, kBatchMaxNP, kSolveThreads);
  if (s.smem > (size_t)kSmemBudget - 64 * 4 - 16) return 0;
  SolveArgs a{};
  a.pop_in = pop_in;
  a.pop_out = pop_out;
  a.fit_out = fit_out;
  a.best_row = best_row;
  a.best_fit = best_fit;
  a.N = c.N;
  a.L = c.L;
  a.K = c.K;
  a.E = c.E;
  a.tour = c.tour;
  a.pc_thresh = c.pc_thresh;
  a.pm_thresh = c.pm_thresh;
  a.seed = c.seed;
  a.gen0 = gen0;
  a.G = G;
  a.NT = s.NT;
  a.MS = s.MS;
  a.XO = s.XO;
  a.NTT = s.NTT;
  a.nblk = s.nblk;
  a.CH = s.CH;
  a.tab = ctx->t32.tab;
  a.own = ctx->t32.own;
  a.bn = ctx->t32.bn;
  a.RS = ctx->t32.RS;
  a.tab_floats = (((int64_t)c.L * c.K * ctx->t32.RS + 3) / 4) * 4;
  a.M32 = ctx->t32.M;
  a.pc32 = ctx->t32.pc;
  a.beta = ctx->beta64;
  a.bnc = ctx->bnc64;
  a.M64 = c.M;
  a.pc64 = ctx->pc;
  a.fin = c.mode == PA_SINR_FINITE_M;
  a.obj = c.objective;
  std::memcpy(args_out, &a, sizeof a);
  return s.smem;
}

// Clusters of size C that can be resident at once for the batched kernel of
// proto's variant with this shared memory (0 when none).
int solve_batch_max_clusters(const pa_ctx* proto, int C, size_t smem) {
  int m = 0;
  if (dispatch_batch(proto, C, 1, nullptr, 0, nullptr, smem, true, &m, nullptr) != cudaSuccess)
    return 0;
  return m;
}

// Persistent batched solve of n instances sharing proto's kernel variant:
// d_args holds their SolveArgs (cluster size C), d_counter must be zero.
cudaError_t launch_solve_batch(const pa_ctx* proto, int C, int clusters, const void* d_args, int n,
                               int* d_counter, size_t smem, cudaStream_t st) {
  return dispatch_batch(proto, C, clusters, static_cast<const SolveArgs*>(d_args), n, d_counter,
                        smem, false, nullptr, st);
}

}  // namespace pa
