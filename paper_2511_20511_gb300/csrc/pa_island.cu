// pa_island.cu -- the PK-means GA (paper Sec. 4.3, Alg. 2): the population is
// partitioned by K-means into C clusters ("islands") and every island
// evolves on its own; the partition is re-applied every few generations
// (Sec. 6.1: every three).
//
// Population K-means (k_island_kmeans, one 1024-thread CTA per call).  A
// chromosome is represented by its one-hot pilot indicators e[u][p] =
// (X[u] == p), one K-vector per user u.  A centroid of m members is
// cnt[u][p] / m with cnt the members' pilot counts, and
//     m^2 |e(n) - cnt/m|^2 = LK m^2 - 2 m S(n) + Q,
//     S(n) = sum_u cnt[u][X_n[u]],      Q = sum_u sum_p cnt[u][p]^2,
// an integer, so the nearest centroid is found exactly: distances of two
// clusters compare by cross-multiplying with the other's m^2 (products below
// 2^62 for N, L*K <= 4096).  Counts live in shared memory (global memory for
// large C*L*K*K); a warp computes one member's S for up to eight clusters at
// a time (lanes over users, then a shuffle sum); the update adds one count
// per (member, user) with shared-memory atomics -- integer sums, so the
// order does not matter.  Initial centroids are C distinct members by a
// partial Fisher-Yates shuffle (Philox tag 4, keyed by the generation);
// Lloyd passes run until no label changes or the pass limit; an emptied
// cluster keeps its counts.
//
// Island lists (k_island_lists): members grouped by island in ascending
// index (off, list) and each member's position in its island (pos), by a
// count, a prefix over islands and warp-level ranks (__match_any_sync).
//
// Island generation (k_island_step, a warp per slot as in k_ga_step): slot
// n of island c at position i is, for i < min(E, m_c), the island's rank-i
// member by (fitness desc, index asc) -- found by i+1 rounds of a warp
// argmax over the island's members -- and otherwise a child of two
// tournaments among the island's members, row-wise crossover and swap
// mutation with the draws of slot n (tag 3), exactly those of k_ga_step.
#include <algorithm>
#include <atomic>

#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int kIslandThreads = 1024;
constexpr int kKmChunk = 8;  // clusters whose sums one warp accumulates at once

struct KmArgs {
  const uint8_t* pop;  // [N][LK]
  int N, L, K, C, max_iter;
  uint64_t seed;
  int gen;
  int32_t* label;      // [N] out
  int32_t* cnt_g;      // [C][LK][K] in global memory, or null (shared memory)
  int32_t* passes;     // [1] out
};

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kIslandThreads) k_island_kmeans(const KmArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_changed;
  const int N = a.N, K = a.K, C = a.C, LK = a.L * a.K;
  const int64_t csz = (int64_t)LK * K;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  unsigned long long* Q = reinterpret_cast<unsigned long long*>(smem);  // [C]
  int* m = reinterpret_cast<int*>(Q + kMaxIslands);                     // [C] centroid sizes
  int* nm = m + kMaxIslands;                                            // [C] new sizes
  int* lab = nm + kMaxIslands;                                          // [N]
  int* idx = lab + kMaxIslandN;                                         // [N]
  int* cnt = a.cnt_g ? a.cnt_g : idx + kMaxIslandN;                     // [C][LK][K]
  const uint8_t* pop = a.pop;

  for (int64_t i = tid; i < C * csz; i += nthr) cnt[i] = 0;
  for (int n = tid; n < N; n += nthr) {
    idx[n] = n;
    lab[n] = -1;
  }
  __syncthreads();
  if (tid == 0) {
    // initial centroids: C distinct members (partial Fisher-Yates shuffle)
    DrawStream ds(a.seed, 0, (uint64_t)a.gen, kTagIsland);
    for (int c = 0; c < C; ++c) {
      const int j = c + (int)below(ds.draw((uint32_t)c), (uint32_t)(N - c));
      const int t = idx[c];
      idx[c] = idx[j];
      idx[j] = t;
      m[c] = 1;
    }
  }
  __syncthreads();
  for (int t = tid; t < C * LK; t += nthr) {
    const int c = t / LK, u = t - c * LK;
    cnt[c * csz + (int64_t)u * K + pop[(int64_t)idx[c] * LK + u]] = 1;
  }
  int passes = 0;
  for (int it = 0; it < a.max_iter; ++it) {
    if (tid < C) Q[tid] = 0ULL;
    if (tid == 0) s_changed = 0;
    __syncthreads();
    for (int64_t i = tid; i < C * csz; i += nthr) {
      const unsigned long long v = (unsigned long long)cnt[i];
      if (v) atomicAdd(&Q[i / csz], v * v);
    }
    __syncthreads();
    // ---- assignment: one warp per member
    for (int n = warp; n < N; n += nwarps) {
      const uint8_t* X = pop + (int64_t)n * LK;
      int best = 0;
      long long bd = 0;
      for (int c0 = 0; c0 < C; c0 += kKmChunk) {
        int s[kKmChunk];
#pragma unroll
        for (int q = 0; q < kKmChunk; ++q) s[q] = 0;
        for (int u = lane; u < LK; u += 32) {
          const int64_t o = (int64_t)u * K + X[u];
#pragma unroll
          for (int q = 0; q < kKmChunk; ++q)
            if (c0 + q < C) s[q] += cnt[(c0 + q) * csz + o];
        }
#pragma unroll
        for (int q = 0; q < kKmChunk; ++q) {
          const int c = c0 + q;
          if (c < C) {
            const long long S = warp_sum_i(s[q]);
            const long long mc = m[c];
            const long long A = (long long)LK * mc * mc - 2 * mc * S + (long long)Q[c];
            const long long mb = m[best];
            if (c == 0 || A * mb * mb < bd * mc * mc) {
              best = c;
              bd = A;
            }
          }
        }
      }
      if (lane == 0) {
        if (lab[n] != best) s_changed = 1;
        lab[n] = best;
      }
    }
    __syncthreads();
    ++passes;
    if (s_changed == 0 || it == a.max_iter - 1) break;
    // ---- update: sizes, then the counts of every cluster that has members
    if (tid < C) nm[tid] = 0;
    __syncthreads();
    for (int n = tid; n < N; n += nthr) atomicAdd(&nm[lab[n]], 1);
    __syncthreads();
    for (int64_t i = tid; i < C * csz; i += nthr)
      if (nm[i / csz] > 0) cnt[i] = 0;
    __syncthreads();
    for (int64_t t = tid; t < (int64_t)N * LK; t += nthr) {
      const int n = (int)(t / LK), u = (int)(t - (int64_t)n * LK);
      atomicAdd(&cnt[lab[n] * csz + (int64_t)u * K + pop[t]], 1);
    }
    if (tid < C && nm[tid] > 0) m[tid] = nm[tid];
    __syncthreads();
  }
  for (int n = tid; n < N; n += nthr) a.label[n] = lab[n];
  if (tid == 0 && a.passes) *a.passes = passes;
}

size_t kmeans_smem(int N, int L, int K, int C, bool cnt_in_smem) {
  size_t b = 8 * (size_t)kMaxIslands + 4 * 2 * (size_t)kMaxIslands + 4 * 2 * (size_t)kMaxIslandN;
  if (cnt_in_smem) b += 4 * (size_t)C * L * K * K;
  (void)N;
  return (b + 15) & ~size_t(15);
}

// Members grouped by island.  One CTA: counts, prefix over islands, then
// chunks of blockDim.x members ranked within warps and across warps.
__global__ void __launch_bounds__(kIslandThreads) k_island_lists(const int32_t* __restrict__ label,
                                                                 int N, int C, int32_t* off,
                                                                 int32_t* list, int32_t* pos) {
  __shared__ int count[kMaxIslands];
  __shared__ int base[kMaxIslands];
  __shared__ int wc[kIslandThreads / 32][kMaxIslands];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < C; c += blockDim.x) count[c] = 0;
  __syncthreads();
  auto lab_of = [&](int n) { return min(max((int)label[n], 0), C - 1); };
  for (int n = tid; n < N; n += blockDim.x) atomicAdd(&count[lab_of(n)], 1);
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int c = 0; c < C; ++c) {
      off[c] = acc;
      base[c] = acc;
      acc += count[c];
    }
    off[C] = acc;
  }
  __syncthreads();
  for (int n0 = 0; n0 < N; n0 += blockDim.x) {
    for (int i = tid; i < (int)(blockDim.x / 32) * C; i += blockDim.x) wc[i / C][i % C] = 0;
    __syncthreads();
    const int n = n0 + tid;
    const int c = n < N ? lab_of(n) : -1 - lane;  // lanes past N form groups of their own
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int rank = __popc(same & ((1u << lane) - 1u));
    if (n < N && rank == 0) wc[warp][c] = __popc(same);
    __syncthreads();
    if (tid < C) {  // prefix of this chunk's warp counts, per island
      int acc = base[tid];
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
        const int t = wc[w][tid];
        wc[w][tid] = acc;
        acc += t;
      }
      base[tid] = acc;
    }
    __syncthreads();
    if (n < N) {
      const int at = wc[warp][c] + rank;
      list[at] = n;
      pos[n] = at - off[c];
    }
    __syncthreads();
  }
}

struct IslandStepArgs {
  const uint8_t* pop;
  const void* fit;
  uint8_t* next;
  const int32_t* label;
  const int32_t* off;
  const int32_t* list;
  const int32_t* pos;
  int N, L, K, C, E, tour;
  uint64_t pc_thresh, pm_thresh, seed;
  int gen;
};

template <typename FT>
__device__ __forceinline__ bool better_vi(FT v, int i, FT bv, int b) {
  if (v > bv) return true;
  if (v < bv) return false;
  return i < b;
}

constexpr int kStepThreads = 256;
constexpr int kStepChildren = kStepThreads / 32;  // one warp per slot

template <typename FT>
__global__ void __launch_bounds__(kStepThreads) k_island_step(const IslandStepArgs a) {
  extern __shared__ uint32_t DR[];  // [kStepChildren][nblk*8]
  __shared__ int chosen[kStepChildren][64];
  const FT* fit = static_cast<const FT*>(a.fit);
  const int64_t LK = (int64_t)a.L * a.K;
  const int T = a.tour;
  const int nblk = (2 * T + 2 + 3 * a.L + 7) / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int n0 = blockIdx.x * kStepChildren; n0 < a.N; n0 += gridDim.x * kStepChildren) {
    const int nc = min(kStepChildren, a.N - n0);
    gen_child_draws(DR, n0, nc, nblk, a.seed, (uint64_t)a.gen, 0);
    __syncthreads();
    if (warp < nc) {
      const int n = n0 + warp;
      const int c = min(max((int)a.label[n], 0), a.C - 1);
      const int base = a.off[c], m = a.off[c + 1] - base, i = a.pos[n];
      const int* mem = a.list + base;
      const int Ec = min(a.E, m);
      uint8_t* __restrict__ child = a.next + n * LK;
      if (i < Ec) {
        // the island's rank-i member: i+1 rounds of a warp argmax
        for (int e = 0; e <= i; ++e) {
          int best = -1;
          FT bv = (FT)0;
          for (int t = lane; t < m; t += 32) {
            const int cand = mem[t];
            bool taken = false;
            for (int f = 0; f < e; ++f) taken |= chosen[warp][f] == cand;
            if (taken) continue;
            const FT v = fit[cand];
            if (best < 0 || better_vi(v, cand, bv, best)) {
              best = cand;
              bv = v;
            }
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const int o = __shfl_xor_sync(0xffffffffu, best, off);
            const FT ov = __shfl_xor_sync(0xffffffffu, bv, off);
            if (o >= 0 && (best < 0 || better_vi(ov, o, bv, best))) {
              best = o;
              bv = ov;
            }
          }
          if (lane == 0) chosen[warp][e] = best;
          __syncwarp();
        }
        const uint8_t* __restrict__ src = a.pop + (int64_t)chosen[warp][i] * LK;
        for (int64_t q = lane; q < LK; q += 32) child[q] = src[q];
      } else {
        const uint32_t* dr = DR + (size_t)warp * nblk * 8;
        int par[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          int best = -1;
          FT bv = (FT)0;
          for (int t = lane; t < T; t += 32) {
            const int cand = mem[below(dr[s * T + t], (uint32_t)m)];
            const FT v = fit[cand];
            if (best < 0 || better_vi(v, cand, bv, best)) {
              best = cand;
              bv = v;
            }
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const int o = __shfl_xor_sync(0xffffffffu, best, off);
            const FT ov = __shfl_xor_sync(0xffffffffu, bv, off);
            if (o >= 0 && (best < 0 || better_vi(ov, o, bv, best))) {
              best = o;
              bv = ov;
            }
          }
          par[s] = best;
        }
        int cut = a.L;
        if ((uint64_t)dr[2 * T] < a.pc_thresh) cut = 1 + (int)below(dr[2 * T + 1], (uint32_t)(a.L - 1));
        const uint8_t* __restrict__ A = a.pop + (int64_t)par[0] * LK;
        const uint8_t* __restrict__ B = a.pop + (int64_t)par[1] * LK;
        const int64_t split = (int64_t)cut * a.K;
        for (int64_t q = lane; q < LK; q += 32) child[q] = q < split ? A[q] : B[q];
        __syncwarp();
        for (int l = lane; l < a.L; l += 32) {
          const int bb = 2 * T + 2 + 3 * l;
          if ((uint64_t)dr[bb] < a.pm_thresh && a.K >= 2) {
            uint8_t* row = child + (int64_t)l * a.K;
            const int i1 = (int)below(dr[bb + 1], (uint32_t)a.K);
            const int jj = (int)below(dr[bb + 2], (uint32_t)(a.K - 1));
            const int i2 = jj + (jj >= i1 ? 1 : 0);
            const uint8_t t = row[i1];
            row[i1] = row[i2];
            row[i2] = t;
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

// Counts of a population K-means fit in shared memory next to the labels.
bool island_cnt_in_smem(int N, int L, int K, int C) {
  return kmeans_smem(N, L, K, C, true) <= (size_t)kSmemBudget;
}

cudaError_t launch_island_kmeans(const pa_ctx* ctx, const uint8_t* pop, int gen, int32_t* labels,
                                 cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  KmArgs a;
  a.pop = pop;
  a.N = c.N;
  a.L = c.L;
  a.K = c.K;
  a.C = c.islands;
  a.max_iter = c.island_iter;
  a.seed = c.seed;
  a.gen = gen;
  a.label = labels;
  a.cnt_g = ctx->isl_cnt;  // null when the counts fit in shared memory
  a.passes = ctx->isl_passes;
  const size_t smem = kmeans_smem(c.N, c.L, c.K, c.islands, a.cnt_g == nullptr);
  static std::atomic<uint64_t> capped{0};
  const uint64_t bit = 1ULL << (ctx->device & 63);
  if (!(capped.load() & bit)) {
    cudaError_t e = raise_smem_cap((const void*)k_island_kmeans, ctx->device);
    if (e != cudaSuccess) return e;
    capped.fetch_or(bit);
  }
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  k_island_kmeans<<<1, kIslandThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_island_lists(const pa_ctx* ctx, const int32_t* labels, const IslandLists& il,
                                cudaStream_t st) {
  (void)cudaGetLastError();
  k_island_lists<<<1, kIslandThreads, 0, st>>>(labels, ctx->cfg.N, ctx->cfg.islands, il.off,
                                               il.list, il.pos);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_island_step(const pa_ctx* ctx, const uint8_t* pop, const void* fit,
                               const int32_t* labels, const IslandLists& il, int32_t gen,
                               uint8_t* next, cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  IslandStepArgs a;
  a.pop = pop;
  a.fit = fit;
  a.next = next;
  a.label = labels;
  a.off = il.off;
  a.list = il.list;
  a.pos = il.pos;
  a.N = c.N;
  a.L = c.L;
  a.K = c.K;
  a.C = c.islands;
  a.E = c.E;
  a.tour = c.tour;
  a.pc_thresh = c.pc_thresh;
  a.pm_thresh = c.pm_thresh;
  a.seed = c.seed;
  a.gen = gen;
  const int blocks = std::max(1, std::min((c.N + kStepChildren - 1) / kStepChildren,
                                          ctx->num_sms * 8));
  const int nblk = (2 * c.tour + 2 + 3 * c.L + 7) / 8;
  const size_t smem = (size_t)kStepChildren * nblk * 32;
  (void)cudaGetLastError();
  if (c.prec == PA_FP64)
    k_island_step<double><<<blocks, kStepThreads, smem, st>>>(a);
  else
    k_island_step<float><<<blocks, kStepThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace pa
