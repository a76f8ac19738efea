// pa_solve_batch.cuh -- the persistent batched solve kernel (many
// instances per launch, a thread-block cluster per instance at a time) and
// its launch dispatch, templated on the column split of the evaluation
// (MAXNP column pairs per thread at most) and the CTA size T:
// pa_solve_batch.cu instantiates the throughput split with 1024-thread CTAs
// (one per SM), pa_solve_batch_lat.cu the one-instance (latency) split,
// pa_solve_batch_small.cu 256-thread CTAs (four instances per SM), as
// separate translation units.
#pragma once

#include <algorithm>
#include <atomic>

#include "pa_solve_body.cuh"

namespace pa {
namespace {

// Many instances per launch (persistent clusters): each cluster takes the
// next instance index from a global counter until the list is exhausted.
// Instances of one launch share the kernel variant (NJ, VEC, FIN, FT); their
// sizes may differ (shared memory is sized for the largest).
template <typename FT, int NJ, int VEC, bool FIN, int THREADS, int MAXNP>
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
    solve_body<FT, NJ, VEC, FIN, MAXNP>(sargs, smem, elites, cluster);
  }
}

}  // namespace

namespace {

template <typename FT, int NJ, int VEC, bool FIN, int THREADS, int MAXNP>
cudaError_t run_solve_batch(int C, int clusters, const SolveArgs* d_args, int n, int* d_counter,
                            size_t smem, bool query_only, int* max_clusters, cudaStream_t st) {
  auto kern = k_solve_batch<FT, NJ, VEC, FIN, THREADS, MAXNP>;
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

template <typename FT, int VEC, bool FIN, int MAXNP, int T>
cudaError_t pick_batch(int NJ, int C, int clusters, const SolveArgs* d, int n, int* ctr,
                       size_t smem, bool q, int* mc, cudaStream_t st) {
  switch (NJ) {
    case 4: return run_solve_batch<FT, 4, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 8: return run_solve_batch<FT, 8, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 12: return run_solve_batch<FT, 12, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 16: return run_solve_batch<FT, 16, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 20: return run_solve_batch<FT, 20, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 24: return run_solve_batch<FT, 24, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 28: return run_solve_batch<FT, 28, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 32: return run_solve_batch<FT, 32, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 36: return run_solve_batch<FT, 36, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 40: return run_solve_batch<FT, 40, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 44: return run_solve_batch<FT, 44, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    case 48: return run_solve_batch<FT, 48, VEC, FIN, T, MAXNP>(C, clusters, d, n, ctr, smem, q, mc, st);
    default: return cudaErrorInvalidValue;
  }
}


template <int MAXNP, int T>
cudaError_t dispatch_batch(const pa_ctx* proto, int C, int clusters, const SolveArgs* d, int n,
                           int* ctr, size_t smem, bool q, int* mc, cudaStream_t st) {
  const pa_config& c = proto->cfg;
  const bool fin = c.mode == PA_SINR_FINITE_M;
  if (c.prec == PA_FP64)
    return run_solve_batch<double, 4, 2, false, T, MAXNP>(C, clusters, d, n, ctr, smem, q,
                                                               mc, st);
  const int NJ = proto->t32.NJ;
  if (proto->t32.vec == 2)
    return fin ? pick_batch<float, 2, true, MAXNP, T>(NJ, C, clusters, d, n, ctr, smem, q, mc, st)
               : pick_batch<float, 2, false, MAXNP, T>(NJ, C, clusters, d, n, ctr, smem, q, mc, st);
  return fin ? pick_batch<float, 1, true, MAXNP, T>(NJ, C, clusters, d, n, ctr, smem, q, mc, st)
             : pick_batch<float, 1, false, MAXNP, T>(NJ, C, clusters, d, n, ctr, smem, q, mc, st);
}

}  // namespace

}  // namespace pa
