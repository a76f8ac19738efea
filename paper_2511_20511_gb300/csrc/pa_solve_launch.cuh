// pa_solve_launch.cuh -- the one-instance cluster kernel (k_solve) and its
// launch, shared by pa_solve.cu (plain GA) and pa_solve_island.cu (island
// mode, Alg. 2), which instantiate it apart so that each translation unit
// stays quick to compile.
#pragma once
#include <cooperative_groups.h>

#include <atomic>

#include "pa_solve_body.cuh"

namespace pa {
namespace {

// One instance per launch: the cluster runs solve_body once.
// ISL: island mode compiled in (Alg. 2; instantiated in pa_solve_island.cu).
template <typename FT, int NJ, int VEC, bool FIN, bool ISL>
__global__ void __launch_bounds__(kSolveThreads) k_solve(const SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int elites[64];
  cg::cluster_group cluster = cg::this_cluster();
  solve_body<FT, NJ, VEC, FIN, kSoloMaxNP, ISL>(a, smem, elites, cluster);
}

template <typename FT, int NJ, int VEC, bool FIN, bool ISL>
cudaError_t run_solve(const SolveArgs& a, const SolveShape& s, bool check_fit, cudaStream_t st) {
  auto kern = k_solve<FT, NJ, VEC, FIN, ISL>;
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
  cfg.gridDim = dim3(s.C, 1, 1);
  cfg.blockDim = dim3(kSolveThreads, 1, 1);
  cfg.dynamicSmemBytes = s.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = s.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (check_fit) {
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess || nclusters < 1) {
      (void)cudaGetLastError();
      return cudaErrorNotSupported;  // this cluster shape cannot be resident
    }
  }
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  e = cudaLaunchKernelEx(&cfg, kern, a);
  count_launch();
  return e;
}

template <typename FT, int VEC, bool FIN, bool ISL>
cudaError_t pick_solve(int NJ, const SolveArgs& a, const SolveShape& s, bool chk, cudaStream_t st) {
  switch (NJ) {
    case 4: return run_solve<FT, 4, VEC, FIN, ISL>(a, s, chk, st);
    case 8: return run_solve<FT, 8, VEC, FIN, ISL>(a, s, chk, st);
    case 12: return run_solve<FT, 12, VEC, FIN, ISL>(a, s, chk, st);
    case 16: return run_solve<FT, 16, VEC, FIN, ISL>(a, s, chk, st);
    case 20: return run_solve<FT, 20, VEC, FIN, ISL>(a, s, chk, st);
    case 24: return run_solve<FT, 24, VEC, FIN, ISL>(a, s, chk, st);
    case 28: return run_solve<FT, 28, VEC, FIN, ISL>(a, s, chk, st);
    case 32: return run_solve<FT, 32, VEC, FIN, ISL>(a, s, chk, st);
    case 36: return run_solve<FT, 36, VEC, FIN, ISL>(a, s, chk, st);
    case 40: return run_solve<FT, 40, VEC, FIN, ISL>(a, s, chk, st);
    case 44: return run_solve<FT, 44, VEC, FIN, ISL>(a, s, chk, st);
    case 48: return run_solve<FT, 48, VEC, FIN, ISL>(a, s, chk, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Island-mode launch (pa_solve_island.cu): `args` a SolveArgs, `shape` a
// SolveShape of this header; FP64, or FP32 with float2 tables.
// cudaErrorNotSupported for other tables.
cudaError_t solve_island_dispatch(const void* args, const void* shape, bool check_fit, bool f64,
                                  int vec, bool fin, int NJ, cudaStream_t st);

}  // namespace pa
