// pa_island.cu -- the PK-means GA (paper Sec. 4.3, Alg. 2): the population is
// partitioned by K-means into C clusters ("islands") and every island
// evolves on its own; the partition is re-applied every few generations
// (Sec. 6.1: every three).
//
// Population K-means.  A chromosome is represented by its one-hot pilot
// indicators e[u][p] = (X[u] == p), one K-vector per user u.  A centroid of
// m members is cnt[u][p] / m with cnt the members' pilot counts, and
//     m^2 |e(n) - cnt/m|^2 = LK m^2 - 2 m S(n) + Q,
//     S(n) = sum_u cnt[u][X_n[u]],      Q = sum_u sum_p cnt[u][p]^2,
// an integer, so the nearest centroid is found exactly: distances of two
// clusters compare by cross-multiplying with the other's m^2 (products below
// 2^62 for N, L*K <= 4096).  The population is staged transposed (a word per
// member and four users, pilots clamped below K); counts are packed 16-bit
// pairs (one load serves two clusters); a lane takes one member, warps
// split the users when the members are few (device code in
// pa_island_kmeans.cuh).  Counts and Q are updated from the members that
// changed cluster (Q from the values the atomics return).  Initial
// centroids are C distinct members by a partial Fisher-Yates shuffle
// (Philox tag 4, keyed by the generation); Lloyd passes run until no label
// changes or the pass limit; an emptied cluster keeps its counts.
// k_island_kmeans_cl runs it on a cluster of up to eight CTAs when counts
// and population fit in shared memory (each CTA assigns a slice of the
// members and replays every CTA's changed members into its own copy of the
// counts); k_island_kmeans on one CTA otherwise (counts in global memory
// for large C*L*K*K, rows read from global memory for large N*L*K).

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
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "pa_island_kmeans.cuh"

namespace pa {
namespace {

constexpr int kIslandThreads = 1024;

struct KmArgs {
  const uint8_t* pop;  // [N][LK]
  int N, L, K, C, max_iter;
  uint64_t seed;
  int gen;
  int32_t* label;      // [N] out
  uint32_t* cnt_g;     // [LK*K][CWp] in global memory, or null (shared memory)
  int32_t* passes;     // [1] out
  int us;              // warps sharing a group of 32 members, each a range of users
  int CWp;             // words per (user, pilot) entry: ceil(C/2), rounded up to odd
  int NP;              // word stride of the staged population (odd)
  int o_cnt, o_sb, o_pw;  // dynamic shared-memory offsets (bytes)
};

// Shared-memory layout of one K-means launch: labels and the initial
// permutation, counts (when in shared memory), per-split partial sums (when
// us > 1), the population staged as words (when it fits).
struct KmLayout {
  int CWp, NP, W, us;
  size_t o_cnt, o_sb, o_pw, total;
};

KmLayout km_layout(int N, int L, int K, int C, bool cnt_in_smem, bool pop_in_smem, int us) {
  KmLayout k;
  const size_t LK = (size_t)L * K;
  k.CWp = ((C + 1) / 2) | 1;
  k.NP = N | 1;
  k.W = (int)((LK + 3) / 4);
  k.us = us;
  size_t b = 2 * 4 * (size_t)((N + 3) & ~3);
  k.o_cnt = b;
  if (cnt_in_smem) b += 4 * LK * K * k.CWp;
  k.o_sb = b;
  if (us > 1) b += 4 * (size_t)us * C * N;
  b = (b + 15) & ~size_t(15);
  k.o_pw = b;
  if (pop_in_smem) b += 4 * (size_t)k.W * k.NP;
  k.total = (b + 15) & ~size_t(15);
  return k;
}

constexpr size_t kKmSmemBudget = (size_t)kSmemBudget - 4096;  // beside the static arrays

// Every loop below is a nested 32-bit loop (counts and members stay below
// 2^24 entries: L*K*K*CWp and N*L*K for N, L*K <= 4096).
//
// Counts are updated, not rebuilt: a pass moves the one-hot vectors of the
// members whose cluster changed (subtracted from the old cluster, added to
// the new), and Q follows each count's change exactly ((v+1)^2 - v^2 =
// 2v + 1 from the value an atomic returns; any order of the moves gives the
// same Q).  This equals the recount over the new partition because a
// cluster's counts are the sum over its current members, except for
// clusters that had no members (kept counts; the initial one-hot centroids):
// those restart from zero when they gain members -- all of which then moved
// in -- and keep their counts while they stay empty.
template <bool CS, bool PS>
__global__ void __launch_bounds__(kIslandThreads) k_island_kmeans(const KmArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long Q[kMaxIslands];
  __shared__ int m[kMaxIslands];       // centroid sizes
  __shared__ int nm[kMaxIslands];      // sizes of the new partition
  __shared__ int live[kMaxIslands];    // the cluster has members in the new partition
  __shared__ int stale[kMaxIslands];   // its counts are not the sum over its members
  __shared__ uint32_t rdraw[kMaxIslands];
  __shared__ int nchg[2];              // members that changed cluster, per pass parity
  const int N = a.N, K = a.K, C = a.C, LK = a.L * a.K, LKK = LK * a.K;
  const int CW = (C + 1) >> 1, CWp = a.CWp, NP = a.NP, W = (LK + 3) >> 2, us = a.us;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const unsigned full = 0xffffffffu;
  int* lab = reinterpret_cast<int*>(smem);  // [N]
  // [N]: the initial permutation, then per pass the changed members
  // (member << 7 | old cluster + 1)
  int* chg = lab + ((N + 3) & ~3);
  uint32_t* cnt = CS ? reinterpret_cast<uint32_t*>(smem + a.o_cnt) : a.cnt_g;
  int* sb = reinterpret_cast<int*>(smem + a.o_sb);            // [us][C][N]
  uint32_t* pw = reinterpret_cast<uint32_t*>(smem + a.o_pw);  // [W][NP]
  if (warp == nwarps - 1) {
    // the initial draws (a Philox block per eight) overlap the set-up below
    for (int c = lane; c < C; c += 32) {
      DrawStream ds(a.seed, 0, (uint64_t)a.gen, kTagIsland);
      rdraw[c] = below(ds.draw((uint32_t)c), (uint32_t)(N - c));
    }
  } else {
    const int sw = nwarps - 1, st = nthr - 32;
    if (PS) {  // word w of member n holds the pilots of users 4w .. 4w+3
      for (int n = warp; n < N; n += sw) {
        const uint8_t* X = a.pop + (int64_t)n * LK;
        for (int w = lane; w < W; w += 32) {
          uint32_t v = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int u = 4 * w + j;
            v |= (uint32_t)(u < LK ? min((int)X[u], K - 1) : K - 1) << (8 * j);
          }
          pw[w * NP + n] = v;
        }
      }
    }
    for (int i = tid; i < LKK * CWp; i += st) cnt[i] = 0;
    for (int n = tid; n < N; n += st) {
      chg[n] = n;
      lab[n] = -1;
    }
    if (tid < kMaxIslands) {
      Q[tid] = 0ULL;
      nm[tid] = 0;
      stale[tid] = 1;
    }
    if (tid < 2) nchg[tid] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    // initial centroids: C distinct members (partial Fisher-Yates shuffle)
    for (int c = 0; c < C; ++c) {
      const int j = c + (int)rdraw[c];
      const int t = chg[c];
      chg[c] = chg[j];
      chg[j] = t;
      m[c] = 1;
    }
  }
  __syncthreads();
  for (int c = warp; c < C; c += nwarps) {  // one-hot of each initial member
    const int n = chg[c], h = (c & 1) * 16;
    unsigned long long dq = 0;
    for (int u = lane; u < LK; u += 32) {
      const int x = km_pilot<PS>(pw, NP, a.pop, LK, K, n, u);
      const uint32_t o = atomicAdd(cnt + (u * K + x) * CWp + (c >> 1), 1u << h);
      dq += (unsigned long long)(2 * km_half(o, h) + 1);
    }
    dq = warp_sum_u64(dq);
    if (lane == 0) atomicAdd(&Q[c], dq);
  }
  __syncthreads();
  const int G = (N + 31) >> 5;
  const int wblk = max(1, 65535 / (4 * N));
  // one member's nearest centroid so far (lowest index on ties)
  auto fold = [&](int c, long long S, int& best, long long& bd) {
    const long long mc = m[c];
    const long long A = (long long)LK * mc * mc - 2 * mc * S + (long long)Q[c];
    const long long mb = m[best];
    if (c == 0 || A * mb * mb < bd * mc * mc) {
      best = c;
      bd = A;
    }
  };
  // a warp's members take their labels (lanes past N pass): changed members
  // are listed, sizes counted by one atomic per distinct label in the warp
  auto record = [&](int n, int best, int par) {
    const bool valid = n < N;
    const int old = valid ? lab[n] : 0;
    const bool moved = valid && old != best;
    const unsigned bm = __ballot_sync(full, moved);
    if (bm) {
      const int leader = __ffs(bm) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&nchg[par], __popc(bm));
      base = __shfl_sync(full, base, leader);
      if (moved) chg[base + __popc(bm & ((1u << lane) - 1u))] = (n << 7) | (old + 1);
    }
    const unsigned same = __match_any_sync(full, valid ? best : -1 - lane);
    if (valid) {
      lab[n] = best;
      if ((int)(__ffs(same) - 1) == lane) atomicAdd(&nm[best], __popc(same));
    }
  };
  int passes = 0;
  for (int it = 0; it < a.max_iter; ++it) {
    const int par = it & 1;
    // ---- assignment: a lane per member, warps over (member group, user range)
    for (int t = warp; t < G * us; t += nwarps) {
      const int g = t / us, s = t - g * us;
      const int n = g * 32 + lane;
      const int nn = n < N ? n : N - 1;
      const int w0 = W * s / us, w1 = W * (s + 1) / us;
      int best = 0;
      long long bd = 0;
      for (int c0 = 0; c0 < C; c0 += 2 * kKmMaxW) {
        int S[2 * kKmMaxW];
        const int i0 = c0 >> 1;
        switch (min(kKmMaxW, CW - i0)) {
#define PA_KM_CASE(NW)                                                                    \
  case NW:                                                                                \
    km_sums<NW, PS>(S, cnt, CWp, i0, K, LK, w0, w1, wblk, pw, NP, a.pop, nn);             \
    break;
          PA_KM_CASE(1)
          PA_KM_CASE(2)
          PA_KM_CASE(3)
          PA_KM_CASE(4)
          PA_KM_CASE(5)
          PA_KM_CASE(6)
          PA_KM_CASE(7)
          default:
            km_sums<8, PS>(S, cnt, CWp, i0, K, LK, w0, w1, wblk, pw, NP, a.pop, nn);
#undef PA_KM_CASE
        }
#pragma unroll
        for (int q = 0; q < 2 * kKmMaxW; ++q) {
          const int c = c0 + q;
          if (c < C) {
            if (us > 1) {
              if (n < N) sb[(s * C + c) * N + n] = S[q];
            } else {
              fold(c, S[q], best, bd);
            }
          }
        }
      }
      if (us == 1) record(n, best, par);
    }
    __syncthreads();
    if (us > 1) {  // the splits' partial sums, then the nearest centroid
      for (int n0 = warp * 32; n0 < N; n0 += nthr) {
        const int n = n0 + lane;
        int best = 0;
        long long bd = 0;
        if (n < N)
          for (int c = 0; c < C; ++c) {
            int S = 0;
            for (int s = 0; s < us; ++s) S += sb[(s * C + c) * N + n];
            fold(c, S, best, bd);
          }
        record(n, best, par);
      }
      __syncthreads();
    }
    ++passes;
    if (nchg[par] == 0 || it == a.max_iter - 1) break;
    // ---- update: clusters that gain members after having none restart at zero
    for (int e = tid; e < LKK; e += nthr)
      for (int i = 0; i < CW; ++i) {
        const bool z0 = stale[2 * i] && nm[2 * i] > 0;
        const bool z1 = 2 * i + 1 < C && stale[2 * i + 1] && nm[2 * i + 1] > 0;
        if (z0 || z1) cnt[e * CWp + i] &= (z0 ? 0u : 0xffffu) | (z1 ? 0u : 0xffff0000u);
      }
    if (tid < C) {
      live[tid] = nm[tid] > 0;
      if (nm[tid] > 0) {
        if (stale[tid]) Q[tid] = 0ULL;
        m[tid] = nm[tid];
      }
    }
    if (tid == 0) nchg[par ^ 1] = 0;
    __syncthreads();
    // ... then every changed member's one-hot moves from its old cluster (when
    // that one still has members) to its new one
    for (int k = warp; k < nchg[par]; k += nwarps) {
      const int e = chg[k], n = e >> 7, A = (e & 127) - 1, Bc = lab[n];
      const bool sub = A >= 0 && live[A];
      const int hb = (Bc & 1) * 16, ha = (A & 1) * 16;
      uint32_t* pb = cnt + (Bc >> 1);
      uint32_t* pold = cnt + (sub ? A >> 1 : 0);
      unsigned long long dqb = 0, dqa = 0;
      for (int u = lane; u < LK; u += 32) {
        const int o = (u * K + km_pilot<PS>(pw, NP, a.pop, LK, K, n, u)) * CWp;
        const uint32_t ob = atomicAdd(pb + o, 1u << hb);
        dqb += (unsigned long long)(2 * km_half(ob, hb) + 1);
        if (sub) {  // the half is >= 1 (the member is counted in it): no borrow
          const uint32_t oa = atomicAdd(pold + o, 0u - (1u << ha));
          dqa += (unsigned long long)(1 - 2 * km_half(oa, ha));
        }
      }
      dqb = warp_sum_u64(dqb);
      dqa = warp_sum_u64(dqa);
      if (lane == 0) {
        atomicAdd(&Q[Bc], dqb);
        if (sub) atomicAdd(&Q[A], dqa);
      }
    }
    if (tid < C) {
      stale[tid] = nm[tid] == 0;
      nm[tid] = 0;
    }
    __syncthreads();
  }
  for (int n = tid; n < N; n += nthr) a.label[n] = lab[n];
  if (tid == 0 && a.passes) *a.passes = passes;
}

struct KmClArgs {
  KmArgs a;
  int Nr;
  int o_lab, o_chg, o_gchg;
};

// The cluster K-means from a population in global memory.
__global__ void __launch_bounds__(kIslandThreads) k_island_kmeans_cl(const KmClArgs ca) {
  cg::cluster_group cluster = cg::this_cluster();
  const KmArgs& a = ca.a;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ KmShared sh;
  const int N = a.N, K = a.K, LK = a.L * a.K, W = (LK + 3) >> 2, NP = a.NP;
  KmView v;
  v.sh = &sh;
  v.pw = reinterpret_cast<uint32_t*>(smem + a.o_pw);
  v.NP = NP;
  v.cnt = reinterpret_cast<uint32_t*>(smem + a.o_cnt);
  v.CWp = a.CWp;
  v.lab = reinterpret_cast<int*>(smem + ca.o_lab);
  v.perm = v.lab + ((N + 3) & ~3);
  v.chg = reinterpret_cast<int*>(smem + ca.o_chg);
  v.gchg = reinterpret_cast<int*>(smem + ca.o_gchg);
  v.sb = reinterpret_cast<int*>(smem + a.o_sb);
  v.us = a.us;
  v.Nr = ca.Nr;
  const KmParams p{a.N, a.L, a.K, a.C, a.max_iter, a.seed, a.gen};
  uint32_t* pw = v.pw;
  const uint8_t* pop = a.pop;
  // word w of member n holds the pilots of users 4w .. 4w+3
  const int passes = km_cluster(v, p, cluster, [&](int warp, int sw, int lane) {
    for (int n = warp; n < N; n += sw) {
      const uint8_t* X = pop + (int64_t)n * LK;
      for (int w = lane; w < W; w += 32) {
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int u = 4 * w + j;
          x |= (uint32_t)(u < LK ? min((int)X[u], K - 1) : K - 1) << (8 * j);
        }
        pw[w * NP + n] = x;
      }
    }
  });
  const int R = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int n_lo = N * rank / R, n_hi = N * (rank + 1) / R;  // N * R < 2^31
  for (int n = n_lo + (int)threadIdx.x; n < n_hi; n += blockDim.x) a.label[n] = v.lab[n];
  if (rank == 0 && threadIdx.x == 0 && a.passes) *a.passes = passes;
  cluster.sync();  // the other CTAs may still read this CTA's lists
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
  return km_layout(N, L, K, C, true, false, 1).total <= kKmSmemBudget;
}

// Words of the K-means counts: two clusters per word, ceil(C/2) words (odd)
// per (user, pilot).
size_t island_cnt_words(int L, int K, int C) {
  return (size_t)L * K * K * (((C + 1) / 2) | 1);
}

// Cluster form of the K-means (k_island_kmeans_cl): R = min(8, N/32) CTAs,
// each holding the whole population and its own counts.
// cudaErrorNotSupported when it does not apply (fewer than 64 members, a
// layout beyond shared memory, a cluster shape that cannot be resident).
cudaError_t launch_island_kmeans_cl(const pa_ctx* ctx, const uint8_t* pop, int gen, int32_t* labels,
                                    cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  if (c.N < 64) return cudaErrorNotSupported;
  const int R = std::min(8, std::max(2, c.N / 32));  // portable cluster sizes
  const int Nr = (c.N + R - 1) / R;
  const int groups = (Nr + 31) / 32, W = (c.L * c.K + 3) / 4;
  int us = std::max(1, std::min({kKmSplits, kIslandThreads / 32 / groups, W}));
  while (us > 1 && km_cl_layout(c.N, c.L, c.K, c.islands, R, us).total > kKmSmemBudget) --us;
  const KmClLayout k = km_cl_layout(c.N, c.L, c.K, c.islands, R, us);
  if (k.total > kKmSmemBudget) return cudaErrorNotSupported;
  // residency of this shape, once per (device, cluster size, shared memory)
  struct Fit {
    int dev, R;
    size_t smem;
    bool ok;
  };
  static Fit fits[64];
  static std::atomic<int> nfits{0};
  static std::atomic<uint64_t> capped{0};
  const uint64_t bit = 1ULL << (ctx->device & 63);
  if (!(capped.load() & bit)) {
    cudaError_t e = raise_smem_cap((const void*)k_island_kmeans_cl, ctx->device);
    if (e != cudaSuccess) return e;
    capped.fetch_or(bit);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(R, 1, 1);
  cfg.blockDim = dim3(kIslandThreads, 1, 1);
  cfg.dynamicSmemBytes = k.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int known = -1;
  const int nf = std::min(nfits.load(), 64);
  for (int i = 0; i < nf; ++i)
    if (fits[i].dev == ctx->device && fits[i].R == R && fits[i].smem == k.total)
      known = fits[i].ok ? 1 : 0;
  if (known < 0) {
    int nclusters = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&nclusters, k_island_kmeans_cl, &cfg) ==
                        cudaSuccess && nclusters >= 1;
    (void)cudaGetLastError();
    const int i = nfits.fetch_add(1);
    if (i < 64) fits[i] = Fit{ctx->device, R, k.total, ok};
    known = ok ? 1 : 0;
  }
  if (!known) return cudaErrorNotSupported;
  KmClArgs ca;
  KmArgs& a = ca.a;
  a.pop = pop;
  a.N = c.N;
  a.L = c.L;
  a.K = c.K;
  a.C = c.islands;
  a.max_iter = c.island_iter;
  a.seed = c.seed;
  a.gen = gen;
  a.label = labels;
  a.cnt_g = nullptr;
  a.passes = ctx->isl_passes;
  a.us = us;
  a.CWp = ((c.islands + 1) / 2) | 1;
  a.NP = k.NP;
  a.o_cnt = (int)k.o_cnt;
  a.o_sb = (int)k.o_sb;
  a.o_pw = (int)k.o_pw;
  ca.Nr = k.Nr;
  ca.o_lab = (int)k.o_lab;
  ca.o_chg = (int)k.o_chg;
  ca.o_gchg = (int)k.o_gchg;
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_island_kmeans_cl, ca);
  count_launch();
  return e;
}

cudaError_t launch_island_kmeans(const pa_ctx* ctx, const uint8_t* pop, int gen, int32_t* labels,
                                 cudaStream_t st) {
  const pa_config& c = ctx->cfg;
  if (ctx->isl_cnt == nullptr) {  // the cluster form, where it fits and can be resident
    cudaError_t e = launch_island_kmeans_cl(ctx, pop, gen, labels, st);
    if (e != cudaErrorNotSupported) return e;
  }
  const bool cs = ctx->isl_cnt == nullptr;
  const bool ps = km_layout(c.N, c.L, c.K, c.islands, cs, true, 1).total <= kKmSmemBudget;
  // warps per group of 32 members: fill the CTA's warps, within the budget
  const int groups = (c.N + 31) / 32, W = (c.L * c.K + 3) / 4;
  int us = std::max(1, std::min({kKmSplits, kIslandThreads / 32 / groups, W}));
  while (us > 1 && km_layout(c.N, c.L, c.K, c.islands, cs, ps, us).total > kKmSmemBudget) --us;
  const KmLayout k = km_layout(c.N, c.L, c.K, c.islands, cs, ps, us);
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
  a.cnt_g = reinterpret_cast<uint32_t*>(ctx->isl_cnt);
  a.passes = ctx->isl_passes;
  a.us = us;
  a.CWp = k.CWp;
  a.NP = k.NP;
  a.o_cnt = (int)k.o_cnt;
  a.o_sb = (int)k.o_sb;
  a.o_pw = (int)k.o_pw;
  const void* fn = cs ? (ps ? (const void*)k_island_kmeans<true, true>
                            : (const void*)k_island_kmeans<true, false>)
                      : (ps ? (const void*)k_island_kmeans<false, true>
                            : (const void*)k_island_kmeans<false, false>);
  static std::atomic<uint64_t> capped[4];
  const int vi = (cs ? 2 : 0) + (ps ? 1 : 0);
  const uint64_t bit = 1ULL << (ctx->device & 63);
  if (!(capped[vi].load() & bit)) {
    cudaError_t e = raise_smem_cap(fn, ctx->device);
    if (e != cudaSuccess) return e;
    capped[vi].fetch_or(bit);
  }
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  if (cs && ps)
    k_island_kmeans<true, true><<<1, kIslandThreads, k.total, st>>>(a);
  else if (cs)
    k_island_kmeans<true, false><<<1, kIslandThreads, k.total, st>>>(a);
  else if (ps)
    k_island_kmeans<false, true><<<1, kIslandThreads, k.total, st>>>(a);
  else
    k_island_kmeans<false, false><<<1, kIslandThreads, k.total, st>>>(a);
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
