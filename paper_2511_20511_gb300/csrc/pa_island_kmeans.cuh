// pa_island_kmeans.cuh -- device code of the population K-means of the
// island GA (Alg. 2's re-clustering): the count-based assignment helpers
// and the cluster form of the Lloyd iteration, shared by the K-means
// kernels (pa_island.cu) and the fused solve's island mode
// (pa_solve_island.cu), which stage the population differently (from
// global memory, or from the cluster's member records).
#pragma once
#include <cooperative_groups.h>

#include "pa_internal.cuh"

namespace pa {
namespace {

namespace cg = cooperative_groups;

constexpr int kKmMaxW = 8;   // pair words of counts one lane sums at once (16 clusters)
constexpr int kKmSplits = 8; // most warps sharing one group of 32 members (user ranges)
constexpr int kKmClusterMax = 16;  // CTAs of a cluster K-means

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Pilot of user u of member n (a pilot >= K reads as K-1): from the staged
// words (clamped when staged), or from the rows.
template <bool PS>
__device__ __forceinline__ int km_pilot(const uint32_t* pw, int NP, const uint8_t* pop, int LK,
                                        int K, int n, int u) {
  if (PS) return (int)((pw[(u >> 2) * NP + n] >> (8 * (u & 3))) & 0xffu);
  return min((int)pop[(int64_t)n * LK + u], K - 1);
}

// Word w of member n: the (clamped) pilots of users 4w .. 4w+3, low byte
// first; bytes past the row end are K-1.
template <bool PS>
__device__ __forceinline__ uint32_t km_word(const uint32_t* pw, int NP, const uint8_t* pop, int LK,
                                            int K, int n, int w) {
  if (PS) return pw[w * NP + n];
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int u = 4 * w + j;
    v |= (uint32_t)(u < LK ? min((int)pop[(int64_t)n * LK + u], K - 1) : K - 1) << (8 * j);
  }
  return v;
}

// S(n, c) for the 2*NW clusters of pair words i0 .. i0+NW-1 over the users
// of words w0 .. w1-1: a lane sums packed 16-bit pairs (one load serves two
// clusters) for wblk words at a time -- a half stays below 2^16 since each
// count is at most N -- and widens them into S.  Words below wfull hold
// four users each; only the row's last word is checked.
template <int NW, bool PS>
__device__ __forceinline__ void km_sums(int (&S)[2 * kKmMaxW], const uint32_t* cnt, int CWp,
                                        int i0, int K, int LK, int w0, int w1, int wblk,
                                        const uint32_t* pw, int NP, const uint8_t* pop, int n) {
  const int wfull = LK >> 2, KC = K * CWp;
#pragma unroll
  for (int q = 0; q < 2 * NW; ++q) S[q] = 0;
  for (int wb = w0; wb < w1; wb += wblk) {
    const int we = min(w1, wb + wblk);
    uint32_t P[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) P[i] = 0;
    int w = wb;
    for (; w < min(we, wfull); ++w) {
      const uint32_t v = km_word<PS>(pw, NP, pop, LK, K, n, w);
      const uint32_t* row = cnt + 4 * w * KC + i0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t* e = row + j * KC + (int)((v >> (8 * j)) & 0xffu) * CWp;
#pragma unroll
        for (int i = 0; i < NW; ++i) P[i] += e[i];
      }
    }
    for (; w < we; ++w) {  // the row's last, partial word
      const uint32_t v = km_word<PS>(pw, NP, pop, LK, K, n, w);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int u = 4 * w + j;
        if (u < LK) {
          const uint32_t* e = cnt + u * KC + (int)((v >> (8 * j)) & 0xffu) * CWp + i0;
#pragma unroll
          for (int i = 0; i < NW; ++i) P[i] += e[i];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      S[2 * i] += (int)(P[i] & 0xffffu);
      S[2 * i + 1] += (int)(P[i] >> 16);
    }
  }
}

// Half h (0: low, 16: high) of a packed word.
__device__ __forceinline__ long long km_half(uint32_t v, int h) {
  return (long long)((v >> h) & 0xffffu);
}

// The cluster form of the K-means (k_island_kmeans_cl, and the fused
// solve in island mode): CTA r of R assigns members
// [N r / R, N (r+1) / R); every CTA holds the whole staged population and
// its own copy of the counts, Q, m and the initial centroids (all computed
// identically).  A pass: assignment of the own slice, the changed members
// listed per CTA; one cluster barrier; every CTA reads the other CTAs'
// changed lists and cluster sizes (distributed shared memory), decides the
// same stop, and replays all changed members into its counts.  Lists and
// sizes are double-buffered by pass parity, so a CTA can list the next
// pass's changes while another still reads this pass's.
struct KmClLayout {
  int NP, W, us, Nr;
  size_t o_lab, o_chg, o_gchg, o_cnt, o_sb, o_pw, total;
};

KmClLayout km_cl_layout(int N, int L, int K, int C, int R, int us) {
  KmClLayout k;
  const size_t LK = (size_t)L * K;
  const int CWp = ((C + 1) / 2) | 1;
  const size_t N4 = (size_t)((N + 3) & ~3);
  k.NP = N | 1;
  k.W = (int)((LK + 3) / 4);
  k.us = us;
  k.Nr = (N + R - 1) / R;
  size_t b = 0;
  k.o_lab = b;   // [N] labels of the own slice (whole range allocated)
  b += 4 * N4;   // + [N] initial permutation
  b += 4 * N4;
  k.o_chg = b;   // [2][N] own changed members per pass parity
  b += 4 * 2 * N4;
  k.o_gchg = b;  // [N] every CTA's changed members of this pass
  b += 4 * N4;
  k.o_cnt = b;
  b += 4 * LK * K * CWp;
  k.o_sb = b;
  if (us > 1) b += 4 * (size_t)us * C * k.Nr;
  b = (b + 15) & ~size_t(15);
  k.o_pw = b;
  b += 4 * (size_t)k.W * k.NP;
  k.total = (b + 15) & ~size_t(15);
  return k;
}

// Per-CTA scalars of a cluster K-means (shared memory).
struct KmShared {
  unsigned long long Q[kMaxIslands];   // sum of squared counts per cluster
  int m[kMaxIslands];                  // centroid sizes
  int nm[kMaxIslands];                 // sizes of the new partition (all CTAs)
  int live[kMaxIslands];               // the cluster has members in the new partition
  int stale[kMaxIslands];              // its counts are not the sum over its members
  uint32_t rdraw[kMaxIslands];         // initial-centroid draws
  int nm_own[2][kMaxIslands];          // own slice's sizes, per pass parity
  int nchg_own[2];                     // own slice's changed members, per pass parity
  int cnt_r[kKmClusterMax];            // changed members of each CTA in this pass
};

// Shared-memory arrays of a cluster K-means (KmClLayout).
struct KmView {
  KmShared* sh;
  uint32_t* pw;   // [W][NP] staged pilots (clamped below K), filled by the stage
  int NP;
  uint32_t* cnt;  // [L*K*K][CWp] packed 16-bit count pairs
  int CWp;
  int* lab;       // [N] labels (the own slice's are final at return)
  int* perm;      // [N] initial permutation
  int* chg;       // [2][N4] own changed members per pass parity
  int* gchg;      // [N] every CTA's changed members of a pass
  int* sb;        // [us][C][Nr] partial sums of the user splits
  int us, Nr;
};

struct KmParams {
  int N, L, K, C, max_iter;
  uint64_t seed;
  int gen;
};

// One population K-means on the calling cluster (every CTA calls it, all
// threads); stage(warp, nwarps, lane) fills v.pw, run by warps 0..nwarps-1
// (= all warps but the last, which makes the initial draws meanwhile).
// Returns the number of assignment passes; the labels of CTA r's slice
// [N r / R, N (r+1) / R) are in its v.lab.  The caller keeps the CTAs
// alive (a cluster barrier) while others may still read this CTA's lists.
template <typename Stage>
__device__ __forceinline__ int km_cluster(const KmView& kv, const KmParams& p,
                                          cg::cluster_group& cluster, Stage stage) {
  KmShared& sh = *kv.sh;
  const int R = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int N = p.N, K = p.K, C = p.C, LK = p.L * p.K, LKK = LK * p.K;
  const int CW = (C + 1) >> 1, CWp = kv.CWp, NP = kv.NP, W = (LK + 3) >> 2, us = kv.us;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const unsigned full = 0xffffffffu;
  const int n_lo = N * rank / R, n_hi = N * (rank + 1) / R;  // N * R < 2^31
  const int Nr = kv.Nr;
  int* lab = kv.lab;
  int* perm = kv.perm;
  int* chg = kv.chg;
  int* gchg = kv.gchg;
  uint32_t* cnt = kv.cnt;
  int* sb = kv.sb;
  uint32_t* pw = kv.pw;
  const int N4 = (N + 3) & ~3;
  if (warp == nwarps - 1) {
    for (int c = lane; c < C; c += 32) {
      DrawStream ds(p.seed, 0, (uint64_t)p.gen, kTagIsland);
      sh.rdraw[c] = below(ds.draw((uint32_t)c), (uint32_t)(N - c));
    }
  } else {
    const int st = nthr - 32;
    stage(warp, nwarps - 1, lane);
    for (int i = tid; i < LKK * CWp; i += st) cnt[i] = 0;
    for (int n = tid; n < N; n += st) {
      perm[n] = n;
      lab[n] = -1;
    }
    if (tid < kMaxIslands) {
      sh.Q[tid] = 0ULL;
      sh.stale[tid] = 1;
      sh.nm_own[0][tid] = 0;
      sh.nm_own[1][tid] = 0;
    }
    if (tid < 2) sh.nchg_own[tid] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    for (int c = 0; c < C; ++c) {
      const int j = c + (int)sh.rdraw[c];
      const int t = perm[c];
      perm[c] = perm[j];
      perm[j] = t;
      sh.m[c] = 1;
    }
  }
  __syncthreads();
  for (int c = warp; c < C; c += nwarps) {
    const int n = perm[c], h = (c & 1) * 16;
    unsigned long long dq = 0;
    for (int u = lane; u < LK; u += 32) {
      const int x = km_pilot<true>(pw, NP, nullptr, LK, K, n, u);
      const uint32_t o = atomicAdd(cnt + (u * K + x) * CWp + (c >> 1), 1u << h);
      dq += (unsigned long long)(2 * km_half(o, h) + 1);
    }
    dq = warp_sum_u64(dq);
    if (lane == 0) atomicAdd(&sh.Q[c], dq);
  }
  __syncthreads();
  const int G = (n_hi - n_lo + 31) >> 5;
  const int wblk = max(1, 65535 / (4 * N));
  auto fold = [&](int c, long long S, int& best, long long& bd) {
    const long long mc = sh.m[c];
    const long long A = (long long)LK * mc * mc - 2 * mc * S + (long long)sh.Q[c];
    const long long mb = sh.m[best];
    if (c == 0 || A * mb * mb < bd * mc * mc) {
      best = c;
      bd = A;
    }
  };
  auto record = [&](int n, int best, int par) {
    const bool valid = n < n_hi;
    const int old = valid ? lab[n] : 0;
    const bool moved = valid && old != best;
    const unsigned bm = __ballot_sync(full, moved);
    if (bm) {
      const int leader = __ffs(bm) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&sh.nchg_own[par], __popc(bm));
      base = __shfl_sync(full, base, leader);
      if (moved)
        chg[par * N4 + base + __popc(bm & ((1u << lane) - 1u))] = (n << 13) | ((old + 1) << 6) | best;
    }
    const unsigned same = __match_any_sync(full, valid ? best : -1 - lane);
    if (valid) {
      lab[n] = best;
      if ((int)(__ffs(same) - 1) == lane) atomicAdd(&sh.nm_own[par][best], __popc(same));
    }
  };
  int passes = 0;
  for (int it = 0; it < p.max_iter; ++it) {
    const int par = it & 1;
    // ---- assignment of the own slice
    for (int t = warp; t < G * us; t += nwarps) {
      const int g = t / us, s = t - g * us;
      const int n = n_lo + g * 32 + lane;
      const int nn = n < n_hi ? n : n_hi - 1;
      const int w0 = W * s / us, w1 = W * (s + 1) / us;
      int best = 0;
      long long bd = 0;
      for (int c0 = 0; c0 < C; c0 += 2 * kKmMaxW) {
        int S[2 * kKmMaxW];
        const int i0 = c0 >> 1;
        switch (min(kKmMaxW, CW - i0)) {
#define PA_KM_CASE(NW)                                                                    \
  case NW:                                                                                \
    km_sums<NW, true>(S, cnt, CWp, i0, K, LK, w0, w1, wblk, pw, NP, nullptr, nn);           \
    break;
          PA_KM_CASE(1)
          PA_KM_CASE(2)
          PA_KM_CASE(3)
          PA_KM_CASE(4)
          PA_KM_CASE(5)
          PA_KM_CASE(6)
          PA_KM_CASE(7)
          default:
            km_sums<8, true>(S, cnt, CWp, i0, K, LK, w0, w1, wblk, pw, NP, nullptr, nn);
#undef PA_KM_CASE
        }
#pragma unroll
        for (int q = 0; q < 2 * kKmMaxW; ++q) {
          const int c = c0 + q;
          if (c < C) {
            if (us > 1) {
              if (n < n_hi) sb[(s * C + c) * Nr + (n - n_lo)] = S[q];
            } else {
              fold(c, S[q], best, bd);
            }
          }
        }
      }
      if (us == 1) record(n, best, par);
    }
    __syncthreads();
    if (us > 1) {
      for (int n0 = n_lo + warp * 32; n0 < n_hi; n0 += nthr) {
        const int n = n0 + lane;
        int best = 0;
        long long bd = 0;
        if (n < n_hi)
          for (int c = 0; c < C; ++c) {
            int S = 0;
            for (int s = 0; s < us; ++s) S += sb[(s * C + c) * Nr + (n - n_lo)];
            fold(c, S, best, bd);
          }
        record(n, best, par);
      }
    }
    // ---- every CTA's labels, lists and sizes of this pass are visible
    cluster.sync();
    if (tid < R) sh.cnt_r[tid] = *cluster.map_shared_rank(&sh.nchg_own[par], tid);
    if (tid >= 32 && tid < 32 + C) {
      const int c = tid - 32;
      int v = 0;
      for (int r = 0; r < R; ++r) v += *cluster.map_shared_rank(&sh.nm_own[par][c], r);
      sh.nm[c] = v;
    }
    __syncthreads();
    int total = 0;
    for (int r = 0; r < R; ++r) total += sh.cnt_r[r];
    ++passes;
    if (total == 0 || it == p.max_iter - 1) break;
    // every CTA's changed members, in CTA order
    for (int k = tid; k < total; k += nthr) {
      int r = 0, base = 0;
      while (k >= base + sh.cnt_r[r]) {
        base += sh.cnt_r[r];
        ++r;
      }
      gchg[k] = *cluster.map_shared_rank(chg + par * N4 + (k - base), r);
    }
    for (int e = tid; e < LKK; e += nthr)
      for (int i = 0; i < CW; ++i) {
        const bool z0 = sh.stale[2 * i] && sh.nm[2 * i] > 0;
        const bool z1 = 2 * i + 1 < C && sh.stale[2 * i + 1] && sh.nm[2 * i + 1] > 0;
        if (z0 || z1) cnt[e * CWp + i] &= (z0 ? 0u : 0xffffu) | (z1 ? 0u : 0xffff0000u);
      }
    if (tid < C) {
      sh.live[tid] = sh.nm[tid] > 0;
      if (sh.nm[tid] > 0) {
        if (sh.stale[tid]) sh.Q[tid] = 0ULL;
        sh.m[tid] = sh.nm[tid];
      }
    }
    // the other parity's own lists were last read before this pass's barrier
    if (tid < kMaxIslands) sh.nm_own[par ^ 1][tid] = 0;
    if (tid == 0) sh.nchg_own[par ^ 1] = 0;
    __syncthreads();
    for (int k = warp; k < total; k += nwarps) {
      const int e = gchg[k], n = e >> 13, A = ((e >> 6) & 127) - 1, Bc = e & 63;
      const bool sub = A >= 0 && sh.live[A];
      const int hb = (Bc & 1) * 16, ha = (A & 1) * 16;
      uint32_t* pb = cnt + (Bc >> 1);
      uint32_t* pold = cnt + (sub ? A >> 1 : 0);
      unsigned long long dqb = 0, dqa = 0;
      for (int u = lane; u < LK; u += 32) {
        const int o = (u * K + km_pilot<true>(pw, NP, nullptr, LK, K, n, u)) * CWp;
        const uint32_t ob = atomicAdd(pb + o, 1u << hb);
        dqb += (unsigned long long)(2 * km_half(ob, hb) + 1);
        if (sub) {
          const uint32_t oa = atomicAdd(pold + o, 0u - (1u << ha));
          dqa += (unsigned long long)(1 - 2 * km_half(oa, ha));
        }
      }
      dqb = warp_sum_u64(dqb);
      dqa = warp_sum_u64(dqa);
      if (lane == 0) {
        atomicAdd(&sh.Q[Bc], dqb);
        if (sub) atomicAdd(&sh.Q[A], dqa);
      }
    }
    if (tid < C) sh.stale[tid] = sh.nm[tid] == 0;
    __syncthreads();
  }
  return passes;
}

}  // namespace
}  // namespace pa
