// pa_prep.cu -- per-instance preparation of the fitness tables (runs once at
// pa_create).  Builds, from beta[j][l][k] (Eq. 2 gains, BS index first):
//   * FP64: bnc[j] = (sum_l sum_k beta[j][l][k]) + sigma2/rho, summed l then k
//     ascending -- the pilot-independent part of the finite-M denominator.
//   * FP32: a BS-minor table tab[(l*K + u)*RS + j] = beta[j][l][u] * 2^s with
//     the own-cell entry (j == l) zeroed, so that one row holds the gains of
//     user u of cell l at every BS; own[l*K + u] = beta[l][l][u] * 2^s; and
//     bn[j] = bnc[j] * 2^s.  Scaling by a power of two is exact and leaves
//     every SINR unchanged (it is a ratio of terms of equal degree).
#include "pa_internal.cuh"

namespace pa {
namespace {

// One block per BS j: the row beta[j][.][.] is staged in shared memory with
// coalesced loads, then one thread adds it up in the fixed (l, k) order.
__global__ void __launch_bounds__(256) k_prep_sums(const double* __restrict__ beta, int L, int K,
                                                   double nc, double scale,
                                                   double* __restrict__ bnc,
                                                   float* __restrict__ bn) {
  extern __shared__ double row[];
  const int LK = L * K;
  for (int j = blockIdx.x; j < L; j += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < LK; i += blockDim.x) row[i] = beta[(size_t)j * LK + i];
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int i = 0; i < LK; ++i) b = __dadd_rn(b, row[i]);
      const double v = __dadd_rn(b, nc);
      bnc[j] = v;
      if (bn) bn[j] = __double2float_rn(__dmul_rn(v, scale));
    }
  }
}

__global__ void k_prep_table(const double* __restrict__ beta, int L, int K, int RS, double scale,
                             int64_t total, float* __restrict__ tab, float* __restrict__ own) {
  const int64_t LK = (int64_t)L * K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / RS;
    const int j = (int)(idx - r * RS);
    float v = 0.f;
    if (r < LK) {
      const int l = (int)(r / K), u = (int)(r - (int64_t)l * K);
      if (j < L && j != l) v = __double2float_rn(__dmul_rn(beta[((int64_t)j * L + l) * K + u], scale));
      if (j == 0) own[r] = __double2float_rn(__dmul_rn(beta[((int64_t)l * L + l) * K + u], scale));
    }
    tab[idx] = v;
  }
}

// Column-tiled layout: tile t, row r = l*K + u, column jj holds
// beta[t*JT + jj][l][u] * 2^s (0 for the own cell and past L).
__global__ void k_prep_table_tiled(const double* __restrict__ beta, int L, int K, int JT, int RSt,
                                   int64_t tile_floats, int ntile, double scale,
                                   float* __restrict__ tab, float* __restrict__ own) {
  const int64_t LK = (int64_t)L * K;
  const int64_t total = tile_floats * ntile;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / tile_floats);
    const int64_t rem = idx - (int64_t)t * tile_floats;
    const int64_t r = rem / RSt;
    const int jj = (int)(rem - r * RSt);
    float v = 0.f;
    if (r < LK) {
      const int l = (int)(r / K), u = (int)(r - (int64_t)l * K);
      const int j = t * JT + jj;
      if (jj < JT && j < L && j != l)
        v = __double2float_rn(__dmul_rn(beta[((int64_t)j * L + l) * K + u], scale));
      if (t == 0 && jj == 0)
        own[r] = __double2float_rn(__dmul_rn(beta[((int64_t)l * L + l) * K + u], scale));
    }
    tab[idx] = v;
  }
}

}  // namespace

cudaError_t launch_prep(pa_ctx* ctx) {
  const int L = ctx->cfg.L, K = ctx->cfg.K;
  const bool f32 = ctx->cfg.prec == PA_FP32;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  k_prep_sums<<<L, 256, sizeof(double) * L * K, ctx->stream>>>(
      ctx->beta64, L, K, ctx->nc, ctx->t32.scale, ctx->bnc64, f32 ? ctx->t32.bn : nullptr);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !f32) return e;
  const int64_t rows = (int64_t)L * K;
  if (ctx->t32.streamed) {
    const int64_t total = ctx->t32.tile_floats * ctx->t32.ntile;
    const int64_t blocks = (total + 255) / 256;
    (void)cudaGetLastError();  // drop a stale error of an earlier call
    k_prep_table_tiled<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, ctx->stream>>>(
        ctx->beta64, L, K, ctx->t32.JT, ctx->t32.RSt, ctx->t32.tile_floats, ctx->t32.ntile,
        ctx->t32.scale, ctx->t32.tab, ctx->t32.own);
    count_launch();
    return cudaGetLastError();
  }
  // table storage is padded to a multiple of 4 floats; pad rows are zero
  const int64_t total = ((rows * ctx->t32.RS + 3) / 4) * 4;
  const int64_t blocks = (total + 255) / 256;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  k_prep_table<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, ctx->stream>>>(
      ctx->beta64, L, K, ctx->t32.RS, ctx->t32.scale, total, ctx->t32.tab, ctx->t32.own);
  count_launch();
  return cudaGetLastError();
}

}  // namespace pa
