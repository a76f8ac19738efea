// pa_ga.cu -- GA generation step, K-means population seeding, best-member
// selection and permutation validation (paper Alg. 1, Sec. 1 items 1-2).
//
// Every random decision comes from a Philox4x64-10 draw stream keyed by the
// seed and addressed by (slot, generation, tag), so a child's draws do not
// depend on which thread makes them and the generation is bit-reproducible.
//
// GA generation (one thread per child slot n):
//   slots 0..E-1  the E best members by (fitness desc, index asc), unchanged
//                 (elitism);
//   slot n >= E   parent a = tournament over draws [0, t), parent b over
//                 [t, 2t) (indices uniform with replacement, best fitness
//                 wins, ties to the lower index); with draw 2t < pc_thresh a
//                 cut c = 1 + below(draw 2t+1, L-1), rows < c from a and
//                 rows >= c from b (row-wise one-cut crossover keeps every
//                 row a permutation), else a copy of a; then for each row l,
//                 with draw 2t+2+3l < pm_thresh, swap two distinct positions
//                 chosen by draws 2t+3+3l and 2t+4+3l.
// Seeding (a cluster of blocks per instance, cells split among them; one
// block per instance when instances are seeded in a batch):
//   Lloyd's K-means on the users' positions relative to their own BS
//   (integer mm; exact int64 centroid sums, one FP64 division; nearest
//   centroid with ties to the lower index; an empty cluster keeps its
//   centroid); initial centroids are k distinct users by a partial
//   Fisher-Yates shuffle.  The assignment A*: in each cell, users in order of
//   (distance to own centroid, index) take pilot = label when free, the rest
//   take the free pilots in ascending order.  Member 0 = A*, members
//   1..n_seeded-1 = A* with each row swapped with probability 1/2, the rest
//   uniformly random rows (Fisher-Yates).
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "pa_internal.cuh"

namespace cg = cooperative_groups;

namespace pa {
namespace {

template <typename FT>
__device__ __forceinline__ bool better(const FT* fit, int a, int b) {
  const FT fa = fit[a], fb = fit[b];
  if (fa > fb) return true;
  if (fa < fb) return false;
  return a < b;
}

// Block-wide best index by (fitness desc, index asc) among members not in
// excluded[0..nex).  Result broadcast through *out.  All threads call it.
template <typename FT>
__device__ int block_best(const FT* fit, int N, const int* excluded, int nex, int* red_idx) {
  int best = -1;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    bool skip = false;
    for (int e = 0; e < nex; ++e) skip |= (excluded[e] == i);
    if (skip) continue;
    if (best < 0 || better(fit, i, best)) best = i;
  }
  // warp reduction
  for (int off = 16; off > 0; off >>= 1) {
    const int o = __shfl_down_sync(0xffffffffu, best, off);
    if (o >= 0 && (best < 0 || better(fit, o, best))) best = o;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red_idx[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = -1;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
      const int o = red_idx[w];
      if (o >= 0 && (b < 0 || better(fit, o, b))) b = o;
    }
    red_idx[32] = b;
  }
  __syncthreads();
  const int r = red_idx[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void swap_two(uint8_t* row, int K, uint32_t ui, uint32_t uj) {
  if (K < 2) return;
  const int i = (int)below(ui, (uint32_t)K);
  const int jj = (int)below(uj, (uint32_t)(K - 1));
  const int j = jj + (jj >= i ? 1 : 0);
  const uint8_t t = row[i];
  row[i] = row[j];
  row[j] = t;
}

struct GaArgs {
  const uint8_t* pop;
  const void* fit;
  uint8_t* next;
  int N, L, K, E, tour;
  uint64_t pc_thresh, pm_thresh, seed;
  int gen;
};

// Best of the candidates drawn by draws dr[0 .. T) (indices uniform with
// replacement), by (fitness desc, index asc): the winner does not depend on
// the order the candidates are compared in, so lanes split the work.
template <typename FT>
__device__ __forceinline__ int warp_tournament(const FT* fit, int N, int T, const uint32_t* dr,
                                               int lane) {
  int best = -1;
  for (int t = lane; t < T; t += 32) {
    const int c = (int)below(dr[t], (uint32_t)N);
    if (best < 0 || better(fit, c, best)) best = c;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const int o = __shfl_xor_sync(0xffffffffu, best, off);
    if (o >= 0 && (best < 0 || better(fit, o, best))) best = o;
  }
  return best;
}

constexpr int kGaThreads = 256;
constexpr int kGaChildren = 8;  // child slots per block (one warp each)

// One block per 8 consecutive child slots.  The block first generates all
// their draws (one Philox block per thread) into shared memory, then each
// warp builds one child: tournaments in parallel lanes, the parents' rows
// copied with coalesced byte streams, the per-row swap mutation with one
// lane per row.
template <typename FT>
__global__ void __launch_bounds__(kGaThreads) k_ga_step(const GaArgs a) {
  extern __shared__ uint32_t DR[];  // [kGaChildren][nblk*8]
  __shared__ int elites[64];
  __shared__ int red[33];
  const FT* fit = static_cast<const FT*>(a.fit);
  const int64_t LK = (int64_t)a.L * a.K;
  const int E = a.E, T = a.tour;
  const int nblk = (2 * T + 2 + 3 * a.L + 7) / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int n0 = blockIdx.x * kGaChildren; n0 < a.N; n0 += gridDim.x * kGaChildren) {
    const int nc = min(kGaChildren, a.N - n0);
    if (n0 < E) {
      for (int e = 0; e < E; ++e) {
        const int b = block_best(fit, a.N, elites, e, red);
        if (threadIdx.x == 0) elites[e] = b;
        __syncthreads();
      }
    }
    gen_child_draws(DR, n0, nc, nblk, a.seed, (uint64_t)a.gen, E);
    __syncthreads();
    if (warp < nc) {
      const int n = n0 + warp;
      uint8_t* __restrict__ child = a.next + n * LK;
      if (n < E) {
        const uint8_t* __restrict__ src = a.pop + (int64_t)elites[n] * LK;
        for (int64_t i = lane; i < LK; i += 32) child[i] = src[i];
      } else {
        const uint32_t* dr = DR + (size_t)warp * nblk * 8;
        const int pa_ = warp_tournament(fit, a.N, T, dr, lane);
        const int pb_ = warp_tournament(fit, a.N, T, dr + T, lane);
        int cut = a.L;
        if ((uint64_t)dr[2 * T] < a.pc_thresh) cut = 1 + (int)below(dr[2 * T + 1], (uint32_t)(a.L - 1));
        const uint8_t* __restrict__ A = a.pop + (int64_t)pa_ * LK;
        const uint8_t* __restrict__ B = a.pop + (int64_t)pb_ * LK;
        const int64_t split = (int64_t)cut * a.K;
        for (int64_t i = lane; i < LK; i += 32) child[i] = i < split ? A[i] : B[i];
        __syncwarp();
        for (int l = lane; l < a.L; l += 32) {
          const int base = 2 * T + 2 + 3 * l;
          if ((uint64_t)dr[base] < a.pm_thresh) swap_two(child + (int64_t)l * a.K, a.K, dr[base + 1], dr[base + 2]);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ seeding
struct SeedArgs {
  const int32_t* user_xy;  // [U][2] or null
  const int32_t* bs_xy;    // [L][2] or null
  int L, K, kk, max_iter;
  int N, n_seeded;
  uint64_t seed;
  uint8_t* pop;
  int32_t* labels;      // [U] out (may be null when feat is null)
  double* centroids;    // [kk][2] out
};

__device__ __forceinline__ double dist2(int32_t fx, int32_t fy, double cx, double cy) {
  const double dx = __dsub_rn((double)fx, cx);
  const double dy = __dsub_rn((double)fy, cy);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__device__ void random_row(uint8_t* row, int K, DrawStream& ds, uint32_t first) {
  for (int k = 0; k < K; ++k) row[k] = (uint8_t)k;
  for (int t = 0; t < K - 1; ++t) {
    const int i = K - 1 - t;
    const int j = (int)below(ds.draw(first + t), (uint32_t)(i + 1));
    const uint8_t tmp = row[i];
    row[i] = row[j];
    row[j] = tmp;
  }
}

constexpr int kSeedClusterThreads = 256;  // per CTA of a seeding cluster

// Shared scalars of a seeding block.
struct SeedShared {
  int changed[2];  // K-means: some label changed, by iteration parity (cluster-wide OR)
  int chg_local;   // some label of this block's users changed
};

// Distances of one (user, centroid) pair per thread when the block's
// user x centroid table fits in this many bytes of shared memory.
constexpr int kSeedDistBytes = 32 * 1024;

// K-means seeding (Sec. 3.3) of one instance by a cluster of C blocks
// (C == 1: one block).  Block `rank` owns cells l with l % C == rank: it
// assigns their users, builds their A* rows and writes their rows of every
// member.  Centroid sums are integers (features are integer millimetres),
// so adding the blocks' partial sums in any order gives the oracle's sums:
// every block adds its partial sums into every block's totals (distributed
// shared memory atomics), and after one cluster barrier per iteration each
// block divides its own totals -- the same operands, so the same centroids
// everywhere.  Totals and change flags are double-buffered by iteration
// parity: a buffer is cleared one iteration after it was read.
__device__ __forceinline__ void seed_body(const SeedArgs& a, unsigned char* smem, SeedShared& sh,
                                          int rank, int C, cg::cluster_group& cluster) {
  const int L = a.L, K = a.K, U = L * K, kk = a.kk;
  const int tid = threadIdx.x, nthr = blockDim.x;
  double* cx = reinterpret_cast<double*>(smem);
  double* cy = cx + kk;
  unsigned long long* sx = reinterpret_cast<unsigned long long*>(cy + kk);  // totals [2][kk]
  unsigned long long* sy = sx + 2 * kk;
  unsigned long long* sn = sy + 2 * kk;
  unsigned long long* px = sn + 2 * kk;  // this block's partial sums [kk]
  unsigned long long* py = px + kk;
  unsigned long long* pn = py + kk;
  int* label = reinterpret_cast<int*>(pn + kk);  // [U] (this block's users)
  int* idx = label + U;          // [U] scratch for the initial shuffle
  int32_t* feat = idx + U;       // [U][2] position relative to the own BS
  uint8_t* astar = reinterpret_cast<uint8_t*>(feat + 2 * U);  // [U] (this block's cells)
  uint8_t* rows_scratch = astar + ((U + 15) & ~15);          // [nthr][K]
  double* D = reinterpret_cast<double*>(rows_scratch + ((nthr * K + 15) & ~15));  // [nuser][kk]
  const bool kmeans = a.user_xy != nullptr && a.n_seeded > 0;
  // this block's cells: rank, rank + C, ...; its users are those cells' users
  const int ncell = rank < L ? (L - 1 - rank) / C + 1 : 0;
  const int nuser = ncell * K;
  auto user_of = [&](int i) { return (rank + (i / K) * C) * K + (i % K); };
  const bool pair_threads = (int64_t)nuser * kk * 8 <= kSeedDistBytes;
  // an address in block r's shared memory (this block's own without a cluster)
  auto at_rank = [&](unsigned long long* p, int r) { return C > 1 ? cluster.map_shared_rank(p, r) : p; };
  auto sync_all = [&]() {
    if (C > 1)
      cluster.sync();
    else
      __syncthreads();
  };

  if (kmeans) {
    for (int u = tid; u < U; u += nthr) {
      idx[u] = u;
      label[u] = -1;
      const int l = u / K;
      feat[2 * u] = a.user_xy[2 * u] - a.bs_xy[2 * l];
      feat[2 * u + 1] = a.user_xy[2 * u + 1] - a.bs_xy[2 * l + 1];
    }
    for (int c = tid; c < 2 * kk; c += nthr) {
      sx[c] = 0;
      sy[c] = 0;
      sn[c] = 0;
    }
    for (int c = tid; c < kk; c += nthr) {
      px[c] = 0;
      py[c] = 0;
      pn[c] = 0;
    }
    if (tid == 0) {
      sh.changed[0] = 0;
      sh.changed[1] = 0;
    }
    __syncthreads();
    if (tid == 0) {
      // initial centroids: kk distinct users by a partial Fisher-Yates
      // shuffle (every block draws the same ones)
      DrawStream ds(a.seed, 0, 0, kTagKmeans);
      for (int i = 0; i < kk; ++i) {
        const int j = i + (int)below(ds.draw((uint32_t)i), (uint32_t)(U - i));
        const int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
        cx[i] = (double)feat[2 * idx[i]];
        cy[i] = (double)feat[2 * idx[i] + 1];
      }
    }
    sync_all();  // every block's totals and flags cleared before any remote add
    for (int it = 0; it < a.max_iter; ++it) {
      const int b = it & 1;
      unsigned long long* tx = sx + b * kk;
      unsigned long long* ty = sy + b * kk;
      unsigned long long* tn = sn + b * kk;
      if (tid == 0) sh.chg_local = 0;
      __syncthreads();  // the previous iteration's clears are done
      // ---- assignment of this block's users (nearest centroid, ties to the lower index)
      if (pair_threads) {
        for (int t = tid; t < nuser * kk; t += nthr) {
          const int i = t / kk, c = t - i * kk, u = user_of(i);
          D[t] = dist2(feat[2 * u], feat[2 * u + 1], cx[c], cy[c]);
        }
        __syncthreads();
      }
      for (int i = tid; i < nuser; i += nthr) {
        const int u = user_of(i);
        const int32_t fx = feat[2 * u], fy = feat[2 * u + 1];
        int best = 0;
        double bd;
        if (pair_threads) {
          const double* d = D + i * kk;
          bd = d[0];
          for (int c = 1; c < kk; ++c)
            if (d[c] < bd) {
              bd = d[c];
              best = c;
            }
        } else {
          bd = dist2(fx, fy, cx[0], cy[0]);
          for (int c = 1; c < kk; ++c) {
            const double d = dist2(fx, fy, cx[c], cy[c]);
            if (d < bd) {
              bd = d;
              best = c;
            }
          }
        }
        if (label[u] != best) sh.chg_local = 1;
        label[u] = best;
        atomicAdd(&px[best], (unsigned long long)(long long)fx);
        atomicAdd(&py[best], (unsigned long long)(long long)fy);
        atomicAdd(&pn[best], 1ULL);
      }
      __syncthreads();
      // this block's partial sums go into every block's parity-b totals
      for (int t = tid; t < C * kk; t += nthr) {
        const int r = t / kk, c = t - r * kk;
        if (pn[c]) {
          atomicAdd(at_rank(&tx[c], r), px[c]);
          atomicAdd(at_rank(&ty[c], r), py[c]);
          atomicAdd(at_rank(&tn[c], r), pn[c]);
        }
      }
      if (tid == 0 && sh.chg_local)
        for (int r = 0; r < C; ++r)
          atomicOr(C > 1 ? cluster.map_shared_rank(&sh.changed[b], r) : &sh.changed[b], 1);
      sync_all();
      const bool done = sh.changed[b] == 0 || it == a.max_iter - 1;
      if (!done)  // x and y coordinates by different threads
        for (int t = tid; t < 2 * kk; t += nthr) {
          const int c = t < kk ? t : t - kk;
          if (tn[c] > 0) {
            const double num = (double)(long long)(t < kk ? tx[c] : ty[c]);
            (t < kk ? cx : cy)[c] = __ddiv_rn(num, (double)(long long)tn[c]);
          }
        }
      __syncthreads();
      // clear the parity-b totals and flag (read above; the next remote adds
      // to them come after the next barrier) and the partial sums
      for (int c = tid; c < kk; c += nthr) {
        tx[c] = 0;
        ty[c] = 0;
        tn[c] = 0;
        px[c] = 0;
        py[c] = 0;
        pn[c] = 0;
      }
      if (tid == 0) sh.changed[b] = 0;
      if (done) break;
    }
    // A*: one thread per cell of this block
    for (int j = tid; j < ncell; j += nthr) {
      const int l = rank + j * C;
      int order[kMaxK];
      double dist[kMaxK];
      bool used[kMaxK];
      int deferred[kMaxK];
      for (int k = 0; k < K; ++k) {
        const int u = l * K + k;
        const int c = label[u];
        dist[k] = dist2(feat[2 * u], feat[2 * u + 1], cx[c], cy[c]);
        order[k] = k;
        used[k] = false;
      }
      for (int i = 1; i < K; ++i) {
        const int v = order[i];
        int jj = i - 1;
        while (jj >= 0 && (dist[order[jj]] > dist[v] || (dist[order[jj]] == dist[v] && order[jj] > v))) {
          order[jj + 1] = order[jj];
          --jj;
        }
        order[jj + 1] = v;
      }
      int nd = 0;
      for (int i = 0; i < K; ++i) {
        const int k = order[i];
        const int p = label[l * K + k];
        if (!used[p]) {
          used[p] = true;
          astar[l * K + k] = (uint8_t)p;
        } else {
          deferred[nd++] = k;
        }
      }
      int nf = 0;
      for (int i = 0; i < nd; ++i) {
        while (used[nf]) ++nf;
        used[nf] = true;
        astar[l * K + deferred[i]] = (uint8_t)nf;
      }
    }
    __syncthreads();
    if (a.labels)
      for (int i = tid; i < nuser; i += nthr) a.labels[user_of(i)] = label[user_of(i)];
    if (rank == 0)
      for (int c = tid; c < kk; c += nthr) {
        a.centroids[2 * c] = cx[c];
        a.centroids[2 * c + 1] = cy[c];
      }
  }
  // Members: one thread per (member n, cell l) row of this block's cells,
  // built in a per-thread shared-memory row and written out as K bytes.
  const int ns = kmeans ? a.n_seeded : 0;
  uint8_t* row = rows_scratch + tid * K;
  const int64_t rows = (int64_t)a.N * ncell;
  for (int64_t t = tid; t < rows; t += nthr) {
    const int n = (int)(t / ncell), l = rank + (int)(t - (int64_t)n * ncell) * C;
    DrawStream ds(a.seed, (uint64_t)n, 0, kTagSeed);
    if (n < ns) {
      for (int k = 0; k < K; ++k) row[k] = astar[l * K + k];
      if (n > 0) {
        const uint32_t u_do = ds.draw((uint32_t)(3 * l));
        const uint32_t ui = ds.draw((uint32_t)(3 * l + 1));
        const uint32_t uj = ds.draw((uint32_t)(3 * l + 2));
        if (u_do < 0x80000000u) swap_two(row, K, ui, uj);
      }
    } else {
      random_row(row, K, ds, (uint32_t)(l * (K > 1 ? K - 1 : 0)));
    }
    uint8_t* dst = a.pop + ((int64_t)n * L + l) * K;
    for (int k = 0; k < K; ++k) dst[k] = row[k];
  }
  // remote blocks may still read this block's sums or flags: leave together
  if (C > 1) cluster.sync();
}

// One instance by a cluster (launched with a cluster dimension of gridDim.x).
__global__ void __launch_bounds__(kSeedClusterThreads) k_seed(const SeedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SeedShared sh;
  cg::cluster_group cluster = cg::this_cluster();
  seed_body(a, smem, sh, (int)cluster.block_rank(), (int)cluster.num_blocks(), cluster);
}

// Cluster i (of num_blocks() CTAs, one CTA without a cluster launch) seeds
// instance i of a batch.
__global__ void __launch_bounds__(kSeedClusterThreads) k_seed_batch(
    const SeedArgs* __restrict__ args, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SeedShared sh;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int i = blockIdx.x / C;
  if (i >= n) return;  // whole clusters only: i is uniform within a cluster
  const SeedArgs a = args[i];
  seed_body(a, smem, sh, (int)cluster.block_rank(), C, cluster);
}

// ------------------------------------------------------------------ best member
template <typename FT>
__global__ void __launch_bounds__(1024) k_argbest(const FT* fit, int N, const uint8_t* pop,
                                                  int64_t LK, uint8_t* best_row,
                                                  double* best_fit) {
  __shared__ int red[33];
  const int b = block_best(fit, N, nullptr, 0, red);
  for (int64_t i = threadIdx.x; i < LK; i += blockDim.x) best_row[i] = pop[b * LK + i];
  if (threadIdx.x == 0) *best_fit = (double)fit[b];
}

// ------------------------------------------------------------------ validation
__global__ void k_validate(const uint8_t* pop, int64_t rows, int K, unsigned long long* first_bad,
                           int L) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* row = pop + r * K;
    unsigned long long seen = 0;
    bool ok = true;
    for (int k = 0; k < K; ++k) {
      const int p = row[k];
      if (p >= K) {
        ok = false;
        break;
      }
      const unsigned long long bit = 1ULL << p;
      if (seen & bit) {
        ok = false;
        break;
      }
      seen |= bit;
    }
    if (!ok) atomicMin(first_bad, (unsigned long long)(r / L));
  }
}

}  // namespace

cudaError_t launch_ga_step(const pa_ctx* ctx, const uint8_t* pop, const void* fit, int32_t gen,
                           uint8_t* next, cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  GaArgs a;
  a.pop = pop;
  a.fit = fit;
  a.next = next;
  a.N = c.N;
  a.L = c.L;
  a.K = c.K;
  a.E = c.E;
  a.tour = c.tour;
  a.pc_thresh = c.pc_thresh;
  a.pm_thresh = c.pm_thresh;
  a.seed = c.seed;
  a.gen = gen;
  const int blocks = std::max(1, std::min((c.N + kGaChildren - 1) / kGaChildren,
                                          ctx->num_sms * 8));
  const int nblk = (2 * c.tour + 2 + 3 * c.L + 7) / 8;
  const size_t smem = (size_t)kGaChildren * nblk * 32;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  if (c.prec == PA_FP64)
    k_ga_step<double><<<blocks, kGaThreads, smem, st>>>(a);
  else
    k_ga_step<float><<<blocks, kGaThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

size_t seed_smem(int L, int K, int kk, int threads, int C) {
  const int U = L * K;
  const int nuser = ((L + C - 1) / C) * K;
  const size_t dist = (size_t)nuser * kk * 8 <= (size_t)kSeedDistBytes ? (size_t)nuser * kk * 8 : 0;
  return (size_t)kk * 8 * 11 + (size_t)U * 4 * 4 + (size_t)((U + 15) & ~15) +
         (((size_t)threads * K + 15) & ~size_t(15)) + dist + 16;
}

static SeedArgs seed_args_of(pa_ctx* ctx, uint8_t* pop);

// Seeding of one instance by a cluster of min(L, 16) CTAs (one CTA per cell
// or more cells per CTA); smaller clusters when that one cannot be resident.
cudaError_t launch_seed(pa_ctx* ctx, uint8_t* pop, cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  const SeedArgs a = seed_args_of(ctx, pop);
  static std::atomic<uint64_t> capped{0};  // devices whose cap is raised (bit per device)
  const uint64_t bit = 1ULL << (ctx->device & 63);
  if (!(capped.load() & bit)) {
    cudaError_t e = raise_smem_cap((const void*)k_seed, ctx->device);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_seed, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    capped.fetch_or(bit);
  }
  cudaError_t e = cudaErrorNotSupported;
  for (int C : {16, 8, 4, 2, 1}) {
    if (C > c.L && C > 1) continue;
    if (ctx->seed_C > 0 && C != ctx->seed_C) continue;  // chosen on an earlier call
    const size_t smem = seed_smem(c.L, c.K, c.kmeans_k, kSeedClusterThreads, C);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kSeedClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ctx->seed_C < 0) {
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_seed, &cfg) != cudaSuccess ||
          nclusters < 1) {
        (void)cudaGetLastError();
        continue;
      }
    }
    (void)cudaGetLastError();  // drop a stale error of an earlier call
    e = cudaLaunchKernelEx(&cfg, k_seed, a);
    count_launch();
    if (e == cudaSuccess) ctx->seed_C = C;
    break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t seed_args_bytes() { return sizeof(SeedArgs); }

static SeedArgs seed_args_of(pa_ctx* ctx, uint8_t* pop) {
  const pa_config& c = ctx->cfg;
  SeedArgs a;
  a.user_xy = ctx->has_positions ? ctx->user_xy : nullptr;
  a.bs_xy = ctx->has_positions ? ctx->bs_xy : nullptr;
  a.L = c.L;
  a.K = c.K;
  a.kk = c.kmeans_k;
  a.max_iter = c.kmeans_max_iter;
  a.N = c.N;
  a.n_seeded = c.n_seeded;
  a.seed = c.seed;
  a.pop = pop;
  a.labels = ctx->labels;
  a.centroids = ctx->centroids;
  return a;
}

size_t seed_fill_args(pa_ctx* ctx, void* out, int C) {
  const SeedArgs a = seed_args_of(ctx, ctx->pop[0]);
  std::memcpy(out, &a, sizeof a);
  return seed_smem(ctx->cfg.L, ctx->cfg.K, ctx->cfg.kmeans_k, kSeedClusterThreads, C);
}

int seed_batch_cluster(int n) {
  // clusters of 16 CTAs while the whole batch fits the GPU at once (<= 9
  // instances on 152 SMs), else 8; larger batches run in waves of 4-CTA
  // clusters (each instance's K-means is a latency chain: splitting its
  // cells over CTAs shortens it, and the waves keep every SM busy)
  for (int C : {16, 8})
    if (n * C <= 152) return C;
  return 4;
}

cudaError_t launch_seed_batch(const void* d_args, int n, size_t smem, int C, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  static std::atomic<uint64_t> capped{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ULL << (dev & 63);
  if (!(capped.load() & bit)) {
    e = raise_smem_cap((const void*)k_seed_batch, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_seed_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    capped.fetch_or(bit);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * C), 1, 1);
  cfg.blockDim = dim3(kSeedClusterThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  e = cudaLaunchKernelEx(&cfg, k_seed_batch, static_cast<const SeedArgs*>(d_args), n);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_argbest(const pa_ctx* ctx, const void* fit, const uint8_t* pop,
                           uint8_t* best_row, double* best_fit_dev, cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  const int64_t LK = (int64_t)c.L * c.K;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  if (c.prec == PA_FP64)
    k_argbest<double><<<1, 1024, 0, st>>>(static_cast<const double*>(fit), c.N, pop, LK, best_row,
                                          best_fit_dev);
  else
    k_argbest<float><<<1, 1024, 0, st>>>(static_cast<const float*>(fit), c.N, pop, LK, best_row,
                                         best_fit_dev);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_validate(const pa_ctx* ctx, const uint8_t* pop, int64_t n, int64_t* first_bad,
                            cudaStream_t st) {
  const int64_t rows = n * ctx->cfg.L;
  const int64_t blocks = std::min<int64_t>((rows + 255) / 256, (int64_t)ctx->num_sms * 16);
  if (blocks <= 0) return cudaSuccess;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  k_validate<<<(unsigned)blocks, 256, 0, st>>>(pop, rows, ctx->cfg.K,
                                               reinterpret_cast<unsigned long long*>(first_bad),
                                               ctx->cfg.L);
  count_launch();
  return cudaGetLastError();
}

}  // namespace pa
