// pa_solve_body.cuh -- the whole-GA-run device code shared by the one-instance
// kernel (pa_solve.cu), its island mode (pa_solve_island.cu) and the batched
// kernels (pa_solve_batch.cu): member records, elites, tournaments, crossover
// and mutation around the fused evaluation, the island mode's re-clustering
// and per-island selection, and the per-instance launch shape.
#pragma once

#include <cooperative_groups.h>

#include <algorithm>

#include "pa_eval_device.cuh"
#include "pa_island_kmeans.cuh"

namespace cg = cooperative_groups;

namespace pa {
namespace {

constexpr int kSolveThreads = 1024;
constexpr int kSmallCtaThreads = 256;  // batched CTAs of the four-per-SM shape
constexpr int kSmallE = 8;  // elites found by one warp in registers up to this E

struct SolveArgs {
  const uint8_t* pop_in;  // N*LK, starting population
  uint8_t* pop_out;       // N*LK, final population
  void* fit_out;          // N fitness values of the final population
  uint8_t* best_row;      // LK, or null
  double* best_fit;       // 1, or null
  int N, L, K, E, tour;
  uint64_t pc_thresh, pm_thresh, seed;
  int gen0, G;
  int NT;    // members per CTA
  int MS;    // member record size in shared memory (bytes): X, then INV at XO
  int XO;    // offset of the inverse permutation inside a record
  int NTT;   // members per evaluation pass
  int nblk;  // Philox blocks of draws per child
  int CH;    // children whose draws are staged at once
  // FP32 tables
  const float* tab;
  const float* own;
  const float* bn;
  int RS;
  int64_t tab_floats;
  float M32, pc32;
  // FP64 data
  const double* beta;
  const double* bnc;
  double M64, pc64;
  int fin;
  int obj;  // PA_OBJ_MIN_SINR: smallest SINR instead of the SE sum
  unsigned long long* stamp;  // when given: %globaltimer (ns) once the outputs are complete
  // island mode (Alg. 2) when isl_C >= 2: each member's island, the islands'
  // member lists (off[C+1], list[N], ascending) and each member's position
  // in its island; E <= kSmallE
  const int32_t* isl_label;
  const int32_t* isl_off;
  const int32_t* isl_list;
  const int32_t* isl_pos;
  int isl_C;
  // re-clustering inside the launch (isl_km): K-means of the population at
  // every generation whose counter is a multiple of isl_R, and at the first
  // when isl_fresh (at most isl_iter passes, isl_us user splits; shared
  // memory at the o_k* offsets); the final labels and member lists are
  // written back to isl_label_out, isl_off_out, isl_list_out, isl_pos_out
  int isl_km, isl_R, isl_iter, isl_fresh, isl_us;
  int o_ksh, o_kpw, o_kcnt, o_klab, o_kchg, o_kgchg, o_ksb;
  int32_t* isl_label_out;
  int32_t* isl_off_out;
  int32_t* isl_list_out;
  int32_t* isl_pos_out;
};

template <typename FT>
__device__ __forceinline__ bool better_s(const FT* fit, int a, int b) {
  const FT fa = fit[a], fb = fit[b];
  if (fa > fb) return true;
  if (fa < fb) return false;
  return a < b;
}

// "member i with fitness v is better than member b with fitness bv": higher
// fitness, or not lower (equal or unordered) and a lower index.
template <typename FT>
__device__ __forceinline__ bool better_v(FT v, int i, FT bv, int b) {
  if (v > bv) return true;
  if (v < bv) return false;
  return i < b;
}
__device__ __forceinline__ float shfl_xor_ft(float v, int off) {
  return __shfl_xor_sync(0xffffffffu, v, off);
}
__device__ __forceinline__ double shfl_xor_ft(double v, int off) {
  return __shfl_xor_sync(0xffffffffu, v, off);
}

// The E best members (fitness desc, index asc) of fit[0..N), E <= EMAX, by
// one warp in E rounds of a warp argmax: round e takes the best member not
// chosen in rounds 0..e-1.  Each lane keeps the fitness of
// its members lane, lane+32, ... (up to CACHE of them; larger populations
// re-read the rest), so every round is a register scan and five shuffles.
template <typename FT, int EMAX, int CACHE>
__device__ __forceinline__ void warp_top_e_rounds(const FT* fit, int N, int E, int lane,
                                                  int* out) {
  FT vc[CACHE];
#pragma unroll
  for (int r = 0; r < CACHE; ++r) vc[r] = lane + 32 * r < N ? fit[lane + 32 * r] : (FT)0;
  int chosen[EMAX];
#pragma unroll
  for (int e = 0; e < EMAX; ++e) {
    chosen[e] = -1;
    if (e < E) {
      int best = -1;
      FT bv = (FT)0;
#pragma unroll
      for (int r = 0; r < CACHE; ++r) {
        const int i = lane + 32 * r;
        bool taken = i >= N;
#pragma unroll
        for (int f = 0; f < e; ++f) taken |= chosen[f] == i;
        if (!taken && (best < 0 || better_v(vc[r], i, bv, best))) {
          best = i;
          bv = vc[r];
        }
      }
      for (int i = lane + 32 * CACHE; i < N; i += 32) {
        bool taken = false;
#pragma unroll
        for (int f = 0; f < e; ++f) taken |= chosen[f] == i;
        const FT v = fit[i];
        if (!taken && (best < 0 || better_v(v, i, bv, best))) {
          best = i;
          bv = v;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, best, off);
        const FT ov = shfl_xor_ft(bv, off);
        if (o >= 0 && (best < 0 || better_v(ov, o, bv, best))) {
          best = o;
          bv = ov;
        }
      }
      chosen[e] = best;
    }
  }
  if (lane == 0)
#pragma unroll
    for (int e = 0; e < EMAX; ++e)
      if (e < E) out[e] = chosen[e];
}

// Tournament over draws dr[0 .. T): candidates uniform with replacement,
// the best by (fitness desc, index asc) wins.  Every lane computes it.
template <typename FT>
__device__ __forceinline__ int tournament_lane(const FT* fit, int N, int T, const uint32_t* dr) {
  constexpr int kU = 4;  // candidates fetched together
  int best = -1;
  FT bv = (FT)0;
  for (int t0 = 0; t0 < T; t0 += kU) {
    int c[kU];
    FT v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) c[u] = t0 + u < T ? (int)below(dr[t0 + u], (uint32_t)N) : -1;
#pragma unroll
    for (int u = 0; u < kU; ++u) v[u] = c[u] >= 0 ? fit[c[u]] : (FT)0;
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (c[u] >= 0 && (best < 0 || better_v(v[u], c[u], bv, best))) {
        best = c[u];
        bv = v[u];
      }
  }
  return best;
}

// Tournament among the m members mem[0..m): candidates mem[u*m >> 32] for
// the draws dr[0 .. T), the best by (fitness desc, index asc) wins.  Every
// lane computes it.
template <typename FT>
__device__ __forceinline__ int tournament_list(const FT* fit, const int* mem, int m, int T,
                                               const uint32_t* dr) {
  int best = -1;
  FT bv = (FT)0;
  for (int t = 0; t < T; ++t) {
    const int c = mem[below(dr[t], (uint32_t)m)];
    const FT v = fit[c];
    if (best < 0 || better_v(v, c, bv, best)) {
      best = c;
      bv = v;
    }
  }
  return best;
}

// The E best (fitness desc, index asc) of the m members mem[0..m), E <= m,
// by one warp in E rounds of a warp argmax; out[0..E) by lane 0.
template <typename FT>
__device__ __forceinline__ void warp_top_e_list(const FT* fit, const int* mem, int m, int E,
                                                int lane, int* out) {
  int chosen[kSmallE];
#pragma unroll
  for (int e = 0; e < kSmallE; ++e) {
    chosen[e] = -1;
    if (e < E) {
      int best = -1;
      FT bv = (FT)0;
      for (int t = lane; t < m; t += 32) {
        const int c = mem[t];
        bool taken = false;
#pragma unroll
        for (int f = 0; f < e; ++f) taken |= chosen[f] == c;
        if (taken) continue;
        const FT v = fit[c];
        if (best < 0 || better_v(v, c, bv, best)) {
          best = c;
          bv = v;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, best, off);
        const FT ov = shfl_xor_ft(bv, off);
        if (o >= 0 && (best < 0 || better_v(ov, o, bv, best))) {
          best = o;
          bv = ov;
        }
      }
      chosen[e] = best;
    }
  }
  if (lane == 0)
#pragma unroll
    for (int e = 0; e < kSmallE; ++e)
      if (e < E) out[e] = chosen[e];
}

// Block-wide best member by (fitness desc, index asc), skipping excluded[0..nex).
template <typename FT>
__device__ int block_best_s(const FT* fit, int N, const int* excluded, int nex, int* red) {
  int best = -1;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    bool skip = false;
    for (int e = 0; e < nex; ++e) skip |= (excluded[e] == i);
    if (skip) continue;
    if (best < 0 || better_s(fit, i, best)) best = i;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const int o = __shfl_down_sync(0xffffffffu, best, off);
    if (o >= 0 && (best < 0 || better_s(fit, o, best))) best = o;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const int o = red[w];
      if (o >= 0 && (b < 0 || better_s(fit, o, b))) b = o;
    }
    red[32] = b;
  }
  __syncthreads();
  const int r = red[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void swap2(uint8_t* row, int K, uint32_t ui, uint32_t uj) {
  if (K < 2) return;
  const int i = (int)below(ui, (uint32_t)K);
  const int jj = (int)below(uj, (uint32_t)(K - 1));
  const int j = jj + (jj >= i ? 1 : 0);
  const uint8_t t = row[i];
  row[i] = row[j];
  row[j] = t;
}

// A child's 32-bit word from its parents' words: the first na bytes from
// parent A, the rest from parent B (na <= 0: all B; na >= 4: all A) -- the
// word holding a row-wise crossover cut.
__device__ __forceinline__ uint32_t merge_word(uint32_t a, uint32_t b, int na) {
  if (na >= 4) return a;
  if (na <= 0) return b;
  const uint32_t mask = (1u << (8 * na)) - 1u;
  return (a & mask) | (b & ~mask);
}

// Remote 32-bit load from another CTA's shared memory (distributed shared
// memory): `addr` is a shared::cluster address from mapa.
__device__ __forceinline__ uint32_t ld_dsmem(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint4 ld_dsmem_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}
__device__ __forceinline__ uint32_t dsmem_addr(const void* local, int rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Remote store of one fitness value (shared::cluster address from mapa).
__device__ __forceinline__ void st_dsmem_ft(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" : : "r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_dsmem_ft(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" : : "r"(addr), "d"(v) : "memory");
}

// Column pairs per thread in the fused FP32 evaluation: the largest divisor
// of NJ/2 not above MAXNP; JS = NJ/2 / NP threads share a (member, pilot).
// More threads per pilot finish an evaluation pass sooner (one instance on a
// 16-CTA cluster is latency-bound: MAXNP 2); fewer, longer threads issue
// fewer index and address instructions per table word (batched instances
// with many members per CTA are issue-bound: MAXNP 5).  The sums are the
// same whatever the split.
constexpr int kSoloMaxNP = 2;
constexpr int kBatchMaxNP = 5;
__host__ __device__ constexpr int fused_np(int NJ, int maxnp) {
  int np = maxnp < NJ / 2 ? maxnp : NJ / 2;
  while (np > 1 && (NJ / 2) % np != 0) --np;
  return np < 1 ? 1 : np;
}
__host__ __device__ constexpr int fused_js(int NJ, int maxnp) {
  return (NJ / 2) / fused_np(NJ, maxnp);
}

// Member record in shared memory (MS bytes): the chromosome X (L*K bytes,
// pilot of each user) at offset 0 and its inverse INV (L*K bytes, user of
// each pilot, row by row) at offset XO.  Crossover takes whole rows, so the
// child's INV rows are its parents' INV rows; a swap mutation updates both.
// Re-clustering inside the fused solve (island mode with isl_km): the
// K-means of the cluster's population (each CTA gathers every member's
// pilots from its owner's records), then every member's label and the
// islands' member lists (ascending index) and positions in every CTA.
__device__ __forceinline__ void island_recluster(const SolveArgs& a, unsigned char* smem,
                                              cg::cluster_group& cluster,
                                              const unsigned char* popc, int gen, int* ilab,
                                              int* ipos, int* ilist, int* ioff, int* icnt) {
  const int N = a.N, L = a.L, K = a.K, C = a.isl_C, LK = L * K, NT = a.NT, MS = a.MS;
  const int W = (LK + 3) >> 2, NP = N | 1, N4 = (N + 3) & ~3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int R = (int)cluster.num_blocks();
  KmView kv;
  kv.sh = reinterpret_cast<KmShared*>(smem + a.o_ksh);
  kv.pw = reinterpret_cast<uint32_t*>(smem + a.o_kpw);
  kv.NP = NP;
  kv.cnt = reinterpret_cast<uint32_t*>(smem + a.o_kcnt);
  kv.CWp = ((C + 1) / 2) | 1;
  kv.lab = reinterpret_cast<int*>(smem + a.o_klab);
  kv.perm = kv.lab + N4;
  kv.chg = reinterpret_cast<int*>(smem + a.o_kchg);
  kv.gchg = reinterpret_cast<int*>(smem + a.o_kgchg);
  kv.sb = reinterpret_cast<int*>(smem + a.o_ksb);
  kv.us = a.isl_us;
  kv.Nr = (N + R - 1) / R;
  const KmParams kp{N, L, K, C, a.isl_iter, a.seed, gen};
  uint32_t* pw = kv.pw;
  const uint32_t kmask = (uint32_t)(K - 1) * 0x01010101u;
  km_cluster(kv, kp, cluster, [&](int w0, int sw, int ln) {
    // pilots of users 4w .. 4w+3 of member n: word w of its record (bytes
    // past the row are the record's zero padding, never read as users)
    const int nts = (NT & (NT - 1)) == 0 ? __ffs(NT) - 1 : -1;  // owner by a shift
    for (int n = w0; n < N; n += sw) {
      const int r = nts >= 0 ? n >> nts : n / NT;
      const uint32_t base = dsmem_addr(popc + (n - r * NT) * MS, r);
      for (int w = ln; w < W; w += 32) pw[w * NP + n] = __vminu4(ld_dsmem(base + 4 * w), kmask);
    }
  });
  // every CTA's slice is final (written before the last pass's barrier);
  // member n of CTA r: n < N (r + 1) / R, the smallest such r
  for (int n = tid; n < N; n += blockDim.x) {
    int r = (n * R) / N;  // N * R < 2^31
    while (n >= N * (r + 1) / R) ++r;
    ilab[n] = *cluster.map_shared_rank(kv.lab + n, r);
  }
  for (int c = tid; c < C; c += blockDim.x) icnt[c] = 0;
  __syncthreads();
  for (int n = tid; n < N; n += blockDim.x) atomicAdd(&icnt[ilab[n]], 1);
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int c = 0; c < C; ++c) {
      ioff[c] = acc;
      acc += icnt[c];
    }
    ioff[C] = acc;
  }
  __syncthreads();
  for (int c = warp; c < C; c += nwarps) {
    int run = 0;
    for (int n0 = 0; n0 < N; n0 += 32) {
      const int n = n0 + lane;
      const bool in = n < N && ilab[n] == c;
      const unsigned b = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int r = run + __popc(b & ((1u << lane) - 1u));
        ilist[ioff[c] + r] = n;
        ipos[n] = r;
      }
      run += __popc(b);
    }
  }
  __syncthreads();
}

template <typename FT, int NJ, int VEC, bool FIN, int MAXNP, bool ISL = false>
__device__ __forceinline__ void solve_body(const SolveArgs& a, unsigned char* smem, int* elites,
                                           cg::cluster_group& cluster) {
  const int rank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const int L = a.L, K = a.K, N = a.N, NT = a.NT, MS = a.MS, XO = a.XO;
  const int LK = L * K;
  constexpr bool F64 = sizeof(FT) == 8;
  constexpr int JS = F64 ? 1 : fused_js(NJ, MAXNP);
  constexpr int NPR = NJ / 2;  // column pairs per (member, pilot)

  // ---- carve shared memory
  unsigned char* p = smem;
  float* T = nullptr;
  float* OWN = nullptr;
  float* BN = nullptr;
  if (!F64) {
    T = reinterpret_cast<float*>(p);
    p += 4 * a.tab_floats;
    OWN = reinterpret_cast<float*>(p);
    p += 4 * ((LK + 3) & ~3);
    BN = reinterpret_cast<float*>(p);
    p += 4 * ((L + 3) & ~3);
  }
  // double buffers are addressed as offsets from the shared-memory base
  const int fit_off0 = (int)(p - smem);
  p += sizeof(FT) * ((N + 1) & ~1);
  const int fit_off1 = (int)(p - smem);
  p += sizeof(FT) * ((N + 1) & ~1);
  auto FITp = [&](int b) { return reinterpret_cast<FT*>(smem + (b ? fit_off1 : fit_off0)); };
  double* SE = reinterpret_cast<double*>(p);  // FP64: NTT*LK per-user SE
  float* PART = reinterpret_cast<float*>(p);  // FP32: NTT*K*NPR per-(pilot, pair) SE
  p += F64 ? 8 * (size_t)a.NTT * LK : 4 * (size_t)((a.NTT * K * NPR + 3) & ~3);
  p = smem + (((p - smem) + 15) & ~15);
  const int pop_off0 = (int)(p - smem);
  p += (size_t)NT * MS;
  const int pop_off1 = (int)(p - smem);
  p += (size_t)NT * MS;
  auto POPp = [&](int b) { return smem + (b ? pop_off1 : pop_off0); };
  p = smem + (((p - smem) + 15) & ~15);
  uint32_t* DR = reinterpret_cast<uint32_t*>(p);  // [CH][nblk*8] draws of staged children
  p += (size_t)a.CH * a.nblk * 32;
  // [32][E] elite candidates (value, index) of the large-E search (E > kSmallE
  // only: the space is not reserved otherwise)
  FT* CV = reinterpret_cast<FT*>(p);
  int* CI = reinterpret_cast<int*>(p + sizeof(FT) * 32 * 64);
  // island mode (E <= kSmallE, so the candidates above are not reserved):
  // labels, positions, member lists, offsets, each island's elites
  const bool isl = ISL && a.isl_C >= 2;
  const int iC = a.isl_C;
  int* ilab = reinterpret_cast<int*>(p);
  int* ipos = ilab + ((N + 3) & ~3);
  int* ilist = ipos + ((N + 3) & ~3);
  int* ioff = ilist + ((N + 3) & ~3);
  int* ielite = ioff + ((iC + 4) & ~3);  // [C][kSmallE]

  const int base_n = rank * NT;
  const int nvalid = max(0, min(NT, N - base_n));

  // ---- stage tables and own members (X and its inverse)
  if (!F64) {
    const float4* s4 = reinterpret_cast<const float4*>(a.tab);
    float4* d4 = reinterpret_cast<float4*>(T);
    for (int64_t i = tid; i < a.tab_floats / 4; i += blockDim.x) d4[i] = __ldg(s4 + i);
    for (int i = tid; i < LK; i += blockDim.x) OWN[i] = __ldg(a.own + i);
    if (FIN)
      for (int i = tid; i < L; i += blockDim.x) BN[i] = __ldg(a.bn + i);
  }
  for (int i = tid; i < NT * MS; i += blockDim.x) POPp(0)[i] = 0;
  if (isl) {
    for (int i = tid; i < N; i += blockDim.x) {
      ilab[i] = min(max((int)a.isl_label[i], 0), iC - 1);
      ipos[i] = a.isl_pos[i];
      ilist[i] = a.isl_list[i];
    }
    for (int i = tid; i <= iC; i += blockDim.x) ioff[i] = a.isl_off[i];
  }
  __syncthreads();
  for (int i = tid; i < nvalid * LK; i += blockDim.x) {
    const int c = i / LK, r = i - c * LK;
    POPp(0)[c * MS + r] = a.pop_in[(int64_t)base_n * LK + i];
  }
  __syncthreads();
  for (int i = tid; i < nvalid * L; i += blockDim.x) {
    const int c = i / L, l = i - c * L;
    const uint8_t* x = POPp(0) + c * MS + l * K;
    uint8_t* inv = POPp(0) + c * MS + XO + l * K;
    for (int k = 0; k < K; ++k) {
      const int q = x[k];
      if (q < K) inv[q] = (uint8_t)k;
    }
  }
  __syncthreads();
  const F32Smem sm{T, OWN, BN, L, K, a.RS, a.M32, a.pc32};

  int cur = 0;
  // lane r's CTA r: its two fitness buffers, mapped once (the fitness push)
  uint32_t fitr0 = 0, fitr1 = 0;
  if ((tid & 31) < C) {
    fitr0 = dsmem_addr(FITp(0), tid & 31);
    fitr1 = dsmem_addr(FITp(1), tid & 31);
  }
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int T_ = a.tour, nblk = a.nblk, E = a.E;
  // FP32 evaluation roles: q = member*K + pilot, column-pair share h.  Each
  // half-warp takes 16 consecutive q with one share h, so the 16 rows it
  // reads in a step (distinct users, RS/2 odd; equal users read the same
  // address) fall in distinct banks
  const int q = (tid / (16 * JS)) * 16 + (tid & 15), h = (tid >> 4) % JS;
  const bool one_chunk = nvalid <= a.CH;
  // member m lives in CTA m / NT: a shift when NT is a power of two
  const int nt_shift = (NT & (NT - 1)) == 0 ? __ffs(NT) - 1 : -1;
  const int n_elite_here = isl ? 0 : max(0, min(E - base_n, nvalid));
  const int E_draw = isl ? 0 : E;  // slots below E_draw take no draws (plain elites)
  for (int g = 0;; ++g) {
    FT* fit = FITp(g & 1);
    const unsigned char* popc = POPp(cur);
    // ---- 1. evaluate own members, broadcast their fitness.  When all
    //         children fit in one draw chunk, the threads the evaluation
    //         leaves idle generate this generation's draws meanwhile (draws
    //         do not depend on fitness).
    bool drawn = false;
    for (int c0 = 0; c0 < nvalid; c0 += a.NTT) {
      const int nv = min(a.NTT, nvalid - c0);
      if (!F64) {
        const int eval_threads = ((nv * K + 15) / 16) * 16 * JS;  // threads up to the last q
        if (q < nv * K) {
          const int c = q / K, pp = q - c * K;
          eval_pilot_f32<NJ, VEC, FIN, JS>(sm, popc + (c0 + c) * MS + XO + pp, K, h,
                                           PART + q * NPR + h * (NPR / JS), a.obj != 0);
        } else if (c0 == 0 && one_chunk && g < a.G && eval_threads + 32 <= (int)blockDim.x &&
                   tid >= ((eval_threads + 31) & ~31)) {
          const int t0 = (eval_threads + 31) & ~31;
          gen_child_draws_from(DR, base_n, nvalid, nblk, a.seed, (uint64_t)(a.gen0 + g), E_draw,
                               tid - t0, blockDim.x - t0);
        }
        if (c0 == 0 && one_chunk && eval_threads + 32 <= (int)blockDim.x) drawn = true;
        __syncthreads();
        for (int c = warp; c < nv; c += nwarps) {
          const float f =
              member_value_bounded<16 * NPR>(PART + c * K * NPR, K * NPR, lane, a.obj != 0);
          const int n = base_n + c0 + c;
          if (lane < C) st_dsmem_ft(((g & 1) ? fitr1 : fitr0) + (uint32_t)(sizeof(FT) * n), (FT)f);
        }
      } else {
        for (int i = tid; i < nv * LK; i += blockDim.x) {
          const int c = i / LK, u = i - c * LK, j = u / K, k = u - j * K;
          const unsigned char* rec = popc + (c0 + c) * MS;
          int qq = rec[u];
          qq = qq < K ? qq : K - 1;
          SE[i] = value_user_f64(a.beta, a.bnc, rec + XO, L, K, j, k, qq, a.fin, a.M64, a.pc64,
                                 a.obj, K, 1);
        }
        __syncthreads();
        if (tid < nv) {
          const double s = member_value_f64(SE + tid * LK, L, K, a.obj);
          const int n = base_n + c0 + tid;
          for (int r = 0; r < C; ++r) cluster.map_shared_rank(fit, r)[n] = (FT)s;
        }
      }
      if (c0 + a.NTT < nvalid) __syncthreads();  // the last pass meets the cluster barrier
    }
    // ---- 2. all fitness values and members of generation g are visible
    cluster.sync();
    if (g == a.G) break;
    if (ISL && a.isl_km && ((g == 0 && a.isl_fresh) || (a.gen0 + g) % a.isl_R == 0))
      island_recluster(a, smem, cluster, POPp(cur), a.gen0 + g, ilab, ipos, ilist, ioff, ielite);
    const bool small_e = E <= kSmallE;
    // ---- 3. elites (CTA holding slots below E).  For E <= 8 warp 0 alone
    //         finds them (register lists) and then fills the elite slots while
    //         the other warps build the other children; for larger E every
    //         warp takes a stripe of the population and warp 0 merges.
    if (n_elite_here > 0 && !small_e) {
      const int stripe = (N + nwarps - 1) / nwarps;
      const int lo = warp * stripe, hi = min(N, lo + stripe);
      for (int e = 0; e < E; ++e) {
        int best = -1;
        FT bv = (FT)0;
        for (int i = lo + lane; i < hi; i += 32) {
          bool taken = false;
          for (int f = 0; f < e; ++f) taken |= (CI[warp * E + f] == i);
          if (taken) continue;
          const FT v = fit[i];
          if (best < 0 || better_v(v, i, bv, best)) {
            best = i;
            bv = v;
          }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const int o = __shfl_xor_sync(0xffffffffu, best, off);
          const FT ov = shfl_xor_ft(bv, off);
          if (o >= 0 && (best < 0 || better_v(ov, o, bv, best))) {
            best = o;
            bv = ov;
          }
        }
        if (lane == 0) {
          CI[warp * E + e] = best;
          CV[warp * E + e] = bv;
        }
        __syncwarp();
      }
      __syncthreads();
      if (warp == 0) {
        const int ncand = nwarps * E;
        for (int e = 0; e < E; ++e) {
          int best = -1, slot = -1;
          FT bv = (FT)0;
          for (int i = lane; i < ncand; i += 32) {
            const int ci = CI[i];
            if (ci < 0) continue;
            const FT v = CV[i];
            if (best < 0 || better_v(v, ci, bv, best)) {
              best = ci;
              bv = v;
              slot = i;
            }
          }
          for (int off = 16; off > 0; off >>= 1) {
            const int o = __shfl_xor_sync(0xffffffffu, best, off);
            const FT ov = shfl_xor_ft(bv, off);
            const int os = __shfl_xor_sync(0xffffffffu, slot, off);
            if (o >= 0 && (best < 0 || better_v(ov, o, bv, best))) {
              best = o;
              bv = ov;
              slot = os;
            }
          }
          if (lane == 0) {
            elites[e] = best;
            CI[slot] = -1;  // consumed
          }
          __syncwarp();
        }
      }
      __syncthreads();
    }
    if (isl) {
      // each island's min(E, m_c) best members, a warp per island
      for (int c = warp; c < iC; c += nwarps) {
        const int m = ioff[c + 1] - ioff[c];
        warp_top_e_list<FT>(fit, ilist + ioff[c], m, min(E, m), lane, ielite + c * kSmallE);
      }
      __syncthreads();
    }
    if (n_elite_here > 0 && small_e && warp == 0) {
      if (E <= 2)
        warp_top_e_rounds<FT, 2, 8>(fit, N, E, lane, elites);
      else
        warp_top_e_rounds<FT, kSmallE, 8>(fit, N, E, lane, elites);
      __syncwarp();
    }
    // ---- 4. children of this CTA's slots: warp w builds slots w, w+nwarps, ...
    unsigned char* popn = POPp(cur ^ 1);
    for (int c0 = 0; c0 < nvalid; c0 += a.CH) {
      const int nc = min(a.CH, nvalid - c0);
      if (!(drawn && c0 == 0)) {
        gen_child_draws(DR, base_n + c0, nc, nblk, a.seed, (uint64_t)(a.gen0 + g), E_draw);
        __syncthreads();
      }
      // elite slots of a small E are warp 0's (it found the elites); other
      // slots go round robin to the remaining warps
      const int ne = (small_e && c0 == 0) ? min(n_elite_here, nc) : 0;
      const int w_first = ne > 0 ? 1 : 0;
      const int w_span = nwarps - w_first;
      int i_begin, i_step;
      if (ne > 0 && warp == 0) {
        i_begin = 0;
        i_step = 1;
      } else {
        i_begin = ne + (warp - w_first);
        i_step = w_span;
      }
      const int i_end = (ne > 0 && warp == 0) ? ne : nc;
      for (int i = i_begin; i < i_end; i += i_step) {
        const int slot = c0 + i;
        const int n = base_n + slot;
        const uint32_t* dr = DR + (size_t)i * nblk * 8;
        uint32_t* child = reinterpret_cast<uint32_t*>(popn + slot * MS);
        int pa_, pb_;
        int64_t split;
        bool elite = false;
        if (isl) {
          // slot n belongs to island c at position i: the island's rank-i
          // member for i < min(E, m_c), else a child of two tournaments
          // among the island's members
          const int c = ilab[n], i = ipos[n], m = ioff[c + 1] - ioff[c];
          if (i < min(E, m)) {
            pa_ = pb_ = ielite[c * kSmallE + i];
            split = LK;
            elite = true;
          } else {
            pa_ = tournament_list(fit, ilist + ioff[c], m, T_, dr);
            pb_ = tournament_list(fit, ilist + ioff[c], m, T_, dr + T_);
            int cut = L;
            if ((uint64_t)dr[2 * T_] < a.pc_thresh) cut = 1 + (int)below(dr[2 * T_ + 1], (uint32_t)(L - 1));
            split = (int64_t)cut * K;
          }
        } else if (n < E) {
          pa_ = pb_ = elites[n];
          split = LK;
          elite = true;
        } else {
          pa_ = tournament_lane(fit, N, T_, dr);
          pb_ = tournament_lane(fit, N, T_, dr + T_);
          int cut = L;
          if ((uint64_t)dr[2 * T_] < a.pc_thresh) cut = 1 + (int)below(dr[2 * T_ + 1], (uint32_t)(L - 1));
          split = (int64_t)cut * K;
        }
        // parents' records from their owners, 16 bytes per lane and load
        const int oa = nt_shift >= 0 ? pa_ >> nt_shift : pa_ / NT;
        const int ob = nt_shift >= 0 ? pb_ >> nt_shift : pb_ / NT;
        const uint32_t ra = dsmem_addr(POPp(cur) + (pa_ - oa * NT) * MS, oa);
        const uint32_t rb = dsmem_addr(POPp(cur) + (pb_ - ob * NT) * MS, ob);
        for (int v = lane; v < (MS >> 4); v += 32) {
          const uint4 qa = ld_dsmem_v4(ra + 16 * v), qb = ld_dsmem_v4(rb + 16 * v);
          // bytes below sp from A: the cut in X, and the same cut in INV
          // (16-byte units never straddle XO); only one unit mixes the two
          const int lo = 16 * v, sp = lo >= XO ? XO + (int)split : (int)split;
          uint4 o;
          if (lo + 16 <= sp) {
            o = qa;
          } else if (lo >= sp) {
            o = qb;
          } else {
            o.x = merge_word(qa.x, qb.x, sp - lo);
            o.y = merge_word(qa.y, qb.y, sp - lo - 4);
            o.z = merge_word(qa.z, qb.z, sp - lo - 8);
            o.w = merge_word(qa.w, qb.w, sp - lo - 12);
          }
          reinterpret_cast<uint4*>(child)[v] = o;
        }
        __syncwarp();
        if (!elite) {
          uint8_t* cx = reinterpret_cast<uint8_t*>(child);
          for (int l = lane; l < L; l += 32) {
            const int base = 2 * T_ + 2 + 3 * l;
            if ((uint64_t)dr[base] < a.pm_thresh && K >= 2) {
              const int i1 = (int)below(dr[base + 1], (uint32_t)K);
              const int jj = (int)below(dr[base + 2], (uint32_t)(K - 1));
              const int i2 = jj + (jj >= i1 ? 1 : 0);
              uint8_t* xr = cx + l * K;
              uint8_t* ir = cx + XO + l * K;
              const uint8_t p1 = xr[i1], p2 = xr[i2];
              xr[i1] = p2;
              xr[i2] = p1;
              if (p1 < K) ir[p1] = (uint8_t)i2;
              if (p2 < K) ir[p2] = (uint8_t)i1;
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }
    cur ^= 1;
  }

  // ---- outputs: final population and fitness, best member
  const FT* fit = FITp(a.G & 1);
  for (int i = tid; i < nvalid * LK; i += blockDim.x) {
    const int c = i / LK, r = i - c * LK;
    a.pop_out[(int64_t)base_n * LK + i] = POPp(cur)[c * MS + r];
  }
  FT* fo = static_cast<FT*>(a.fit_out);
  for (int c = tid; c < nvalid; c += blockDim.x) fo[base_n + c] = fit[base_n + c];
  if (rank == 0 && a.best_row && warp == 0) {
    int best = -1;
    FT bv = (FT)0;
    for (int i = lane; i < N; i += 32) {
      const FT v = fit[i];
      if (best < 0 || better_v(v, i, bv, best)) {
        best = i;
        bv = v;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const int o = __shfl_xor_sync(0xffffffffu, best, off);
      const FT ov = shfl_xor_ft(bv, off);
      if (o >= 0 && (best < 0 || better_v(ov, o, bv, best))) {
        best = o;
        bv = ov;
      }
    }
    const uint8_t* src = cluster.map_shared_rank(POPp(cur), best / NT) + (best % NT) * MS;
    for (int r = lane; r < LK; r += 32) a.best_row[r] = src[r];
    if (lane == 0) *a.best_fit = (double)fit[best];
  }
  if (ISL && a.isl_km && rank == 0) {  // the last clustering, for the caller
    for (int i = tid; i < N; i += blockDim.x) {
      a.isl_label_out[i] = ilab[i];
      a.isl_list_out[i] = ilist[i];
      a.isl_pos_out[i] = ipos[i];
    }
    for (int i = tid; i <= iC; i += blockDim.x) a.isl_off_out[i] = ioff[i];
  }
  cluster.sync();  // keep this CTA's shared memory alive for remote readers
  if (a.stamp && rank == 0 && tid == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    *a.stamp = t;
  }
}

// ------------------------------------------------------------------ launch
struct SolveShape {
  int C, NT, MS, XO, NTT, nblk, CH;
  size_t smem;
};

SolveShape solve_shape(const pa_ctx* ctx, int C, int maxnp, int threads) {
  const pa_config& c = ctx->cfg;
  const bool f64 = c.prec == PA_FP64;
  const int LK = c.L * c.K;
  SolveShape s{};
  s.nblk = (2 * c.tour + 2 + 3 * c.L + 7) / 8;
  s.C = C;
  s.NT = (c.N + C - 1) / C;
  s.CH = std::max(1, std::min(s.NT, 16384 / (s.nblk * 32)));
  // record = X | INV, 16-byte aligned halves (records are copied 16 bytes
  // per lane); an odd number of 16-byte units per record spreads the
  // per-member inverse reads of one warp over the banks
  s.XO = ((LK + 15) / 16) * 16;
  s.MS = 2 * s.XO;
  if ((s.MS / 16) % 2 == 0) s.MS += 16;
  const int NJ = ctx->t32.NJ;
  const int JS = f64 ? 1 : fused_js(NJ, maxnp);
  const int NPR = f64 ? 0 : NJ / 2;
  if (f64) {
    s.NTT = std::max(1, std::min(s.NT, 2048 / std::max(1, LK)));
  } else {
    // members per pass: their (member, pilot) pairs, in half-warp groups of
    // 16, times JS shares fit the block
    s.NTT = 0;
    for (int n = s.NT; n >= 1; --n)
      if (((n * c.K + 15) / 16) * 16 * JS <= threads) {
        s.NTT = n;
        break;
      }
    if (s.NTT == 0) {  // one member's pilots need more threads than the CTA has
      s.smem = ~size_t(0);
      return s;
    }
  }
  size_t b = 0;
  if (!f64) {
    const size_t tab = (((size_t)LK * ctx->t32.RS + 3) / 4) * 4;
    b += 4 * tab + 4 * (size_t)((LK + 3) & ~3) + 4 * (size_t)((c.L + 3) & ~3);
  }
  const size_t fsz = f64 ? 8 : 4;
  b += 2 * fsz * (size_t)((c.N + 1) & ~1);
  b += f64 ? 8 * (size_t)s.NTT * LK : 4 * (size_t)((s.NTT * c.K * NPR + 3) & ~3);
  b = (b + 15) & ~size_t(15);
  b += 2 * (size_t)s.NT * s.MS;
  b = (b + 15) & ~size_t(15);
  b += (size_t)s.CH * s.nblk * 32;
  if (c.E > kSmallE) b += (f64 ? 8 : 4) * 32 * 64 + 4 * 32 * 64;  // elite candidates
  if (c.islands >= 2) {  // labels, positions, lists, offsets, island elites
    const size_t N4 = (size_t)((c.N + 3) & ~3);
    b += 4 * (3 * N4 + (size_t)((c.islands + 4) & ~3) + (size_t)c.islands * kSmallE);
  }
  s.smem = (b + 15) & ~size_t(15);
  return s;
}

}  // namespace
}  // namespace pa
