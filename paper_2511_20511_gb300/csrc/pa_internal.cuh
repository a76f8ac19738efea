// pa_internal.cuh -- internal declarations shared by the CUDA sources of
// libpa.so (context layout, kernel launchers, device helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/pa.h"

namespace pa {

// ----------------------------------------------------------------- limits
constexpr int kMaxK = 64;            // pilots per cell (uint8 rows, smem rows)
constexpr int kMaxL = 255;           // cells
constexpr int kMaxNJ = 48;           // widest per-thread BS vector of the FP32 kernel
constexpr int kSmemBudget = 227 * 1024;

// Stream tags of the counter-based generator (counter word 3).
enum : uint32_t { kTagSeed = 1, kTagKmeans = 2, kTagGa = 3, kTagIsland = 4 };

// Islands of the PK-means GA: at most this many clusters and members.
constexpr int kMaxIslands = 64;
constexpr int kMaxIslandN = 4096;

// Prepared FP32 tables of one instance (device pointers, owned by ctx).
struct F32Tables {
  float* tab = nullptr;  // [L*K rows][RS]: row l*K+u, col j: beta[j][l][u]*2^s, 0 if j==l
  float* own = nullptr;  // [L*K]: beta[l][l][u]*2^s
  float* bn = nullptr;   // [L]: (B_j + sigma2/rho) * 2^s
  int RS = 0;            // row stride (floats)
  int NJ = 0;            // BS entries read per row (even, >= L)
  int vec = 1;           // 2: float2 loads (K <= 16), 1: scalar loads
  float M = 0.f;         // antennas
  float pc = 0.f;        // sigma2/(tau_p rho) * 2^s
  int scale_exp = 0;     // s
  double scale = 1.0;    // 2^s
  // column-tiled table for instances whose table exceeds shared memory:
  // ntile tiles of JT BS columns, each [L*K rows][RSt] floats, tile_floats
  // (padded to 4) apart; tab then holds the tiles back to back
  int streamed = 0;
  int JT = 0, ntile = 0, RSt = 0;
  int64_t tile_floats = 0;
  float* partial = nullptr;  // scratch: per-(member, tile) fitness partials
  int64_t partial_cap = 0;   // members it can hold
  int* err_flag = nullptr;   // set by a kernel whose bounded wait gave up
};

// Members of a population grouped by island (device arrays).
struct IslandLists {
  int32_t* off = nullptr;   // [C+1] first position of each island in list
  int32_t* list = nullptr;  // [N] members grouped by island, ascending within
  int32_t* pos = nullptr;   // [N] position of each member within its island
};

}  // namespace pa

struct pa_ctx {
  pa_config cfg{};
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  double nc = 0.0;  // sigma2 / rho
  double pc = 0.0;  // sigma2 / (tau_p rho)
  // instance data (device)
  double* beta64 = nullptr;   // [L][L][K] as given
  double* bnc64 = nullptr;    // [L]: B_j + nc (FP64, oracle order)
  pa::F32Tables t32;
  int32_t* user_xy = nullptr; // [L*K][2] user positions (mm), or null
  int32_t* bs_xy = nullptr;   // [L][2] BS positions (mm), or null
  int32_t* labels = nullptr;  // [L*K]
  double* centroids = nullptr;  // [kmeans_k][2]
  int has_positions = 0;
  // resident population (device)
  uint8_t* pop[2] = {nullptr, nullptr};
  int cur = 0;
  void* fit = nullptr;         // [N] float or double
  int32_t generation = 0;
  int solve_C = -1;            // cluster size of the fused solve kernel (-1: not chosen, 0: none)
  int seed_C = -1;             // cluster size of the seeding kernel (-1: not chosen)
  int wait_check = 0;          // an FP32 evaluation ran since t32.err_flag was last read
  int test_stall = 0;          // PA_FLAG_TEST_STALL_COPIES still pending (one-shot)
  // islands of the PK-means GA (cfg.islands >= 2)
  int32_t* isl_label = nullptr;  // [N] island of each member of the resident population
  pa::IslandLists isl_res;       // member lists of isl_label
  pa::IslandLists isl_usr;       // member lists of a pa_island_step call's labels
  int32_t* isl_cnt = nullptr;    // K-means counts in global memory when they exceed shared memory
  int32_t* isl_passes = nullptr; // [1] assignment passes of the last K-means
  int isl_valid = 0;             // isl_label belongs to the resident population
  void* arena = nullptr;  // the one device allocation the buffers below are carved from
  // scratch
  int64_t* scratch_i64 = nullptr;  // small device scratch (flags, argbest)
  uint8_t* best_row = nullptr;     // [L*K], then the best fitness (double) 8-byte aligned
  uint8_t* h_best = nullptr;       // pinned host copy of the same bytes (first pa_solve)
  // host staging for *_host calls
  uint8_t* stage_pop = nullptr;
  void* stage_fit = nullptr;
  int64_t stage_cap = 0;
  std::string err;
};

namespace pa {

pa_status fail(pa_ctx* ctx, pa_status st, const std::string& msg);
// process-wide count of kernels this library has launched
void count_launch();
pa_status cuda_check(pa_ctx* ctx, cudaError_t e, const char* what);

// ----------------------------------------------------------------- launchers
// pa_prep.cu
cudaError_t launch_prep(pa_ctx* ctx);
// host-side checks of one instance: beta finite and > 0 (returns the largest
// value through bmax), relative positions within int32
bool instance_ok(const pa_config& c, const double* beta, const int32_t* user_xy_mm,
                 const int32_t* bs_xy_mm, double* bmax);
// pa_fitness.cu
cudaError_t launch_eval_f32(pa_ctx* ctx, const uint8_t* pop, int64_t n, float* fit,
                            cudaStream_t st);
cudaError_t launch_eval_f64(const pa_ctx* ctx, const uint8_t* pop, int64_t n, double* fit,
                            cudaStream_t st);
bool f32_supported(int L, int K, size_t* smem_bytes);
// pa_stream.cu: column-tiled evaluation for tables beyond shared memory
bool f32_stream_geometry(int L, int K, int* JT, int* RSt, int* vec, int* ntile);
cudaError_t launch_eval_f32_stream(pa_ctx* ctx, const uint8_t* pop, int64_t n, float* fit,
                                   cudaStream_t st);
// pa_ga.cu
cudaError_t launch_ga_step(const pa_ctx* ctx, const uint8_t* pop, const void* fit, int32_t gen,
                           uint8_t* next, cudaStream_t st);
cudaError_t launch_seed(pa_ctx* ctx, uint8_t* pop, cudaStream_t st);
cudaError_t launch_argbest(const pa_ctx* ctx, const void* fit, const uint8_t* pop,
                           uint8_t* best_row, double* best_fit_dev, cudaStream_t st);
// pa_solve.cu
// isl_label / isl: island mode (Alg. 2) with these labels and member lists;
// isl_km: the re-clustering inside the launch (labels and lists written back)
cudaError_t launch_solve(pa_ctx* ctx, const uint8_t* pop_in, uint8_t* pop_out, int gen0, int G,
                         void* fit_out, uint8_t* best_row, double* best_fit, cudaStream_t st,
                         int32_t* isl_label = nullptr, IslandLists* isl = nullptr,
                         bool isl_km = false);
size_t solve_args_bytes();
// latency: the one-instance kernel's column split (few concurrent
// instances) instead of the throughput split; threads: CTA size, 1024 (one
// CTA per SM) or 256 (four per SM)
size_t solve_fill_args(const pa_ctx* ctx, int C, int gen0, int G, const uint8_t* pop_in,
                       uint8_t* pop_out, void* fit_out, uint8_t* best_row, double* best_fit,
                       void* args_out, bool latency = false, int threads = 1024);
int solve_batch_max_clusters(const pa_ctx* proto, int C, size_t smem, bool latency = false,
                             int threads = 1024);
void solve_args_set_stamp(void* args, unsigned long long* stamp);
cudaError_t launch_solve_batch(const pa_ctx* proto, int C, int clusters, const void* d_args, int n,
                               int* d_counter, size_t smem, cudaStream_t st, bool latency = false,
                               int threads = 1024);
// pa_ga.cu: seed many instances at once (a cluster of C CTAs each) from n
// seed argument records (seed_args_bytes() each, filled by seed_fill_args
// for that C) in device memory; smem = the largest seed_fill_args value
size_t seed_args_bytes();
size_t seed_fill_args(pa_ctx* ctx, void* out, int C);
// cluster size of a batched seeding launch of n instances
int seed_batch_cluster(int n);
cudaError_t launch_seed_batch(const void* d_args, int n, size_t smem, int C, cudaStream_t st);
cudaError_t launch_validate(const pa_ctx* ctx, const uint8_t* pop, int64_t n, int64_t* first_bad,
                            cudaStream_t st);
// pa_island.cu: PK-means GA (Alg. 2)
bool island_cnt_in_smem(int N, int L, int K, int C);
size_t island_cnt_words(int L, int K, int C);
cudaError_t launch_island_kmeans(const pa_ctx* ctx, const uint8_t* pop, int gen, int32_t* labels,
                                 cudaStream_t st);
cudaError_t launch_island_lists(const pa_ctx* ctx, const int32_t* labels, const IslandLists& il,
                                cudaStream_t st);
cudaError_t launch_island_step(const pa_ctx* ctx, const uint8_t* pop, const void* fit,
                               const int32_t* labels, const IslandLists& il, int32_t gen,
                               uint8_t* next, cudaStream_t st);

// Raise a kernel's dynamic shared-memory cap to what the device allows
// beside the kernel's static shared memory (call once per kernel and device).
inline cudaError_t raise_smem_cap(const void* fn, int dev) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

// ----------------------------------------------------------------- device helpers
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x64
// S-box, Weyl key schedule.
struct Philox4x64 {
  uint64_t v[4];
};

__device__ __forceinline__ Philox4x64 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                    uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  Philox4x64 o;
  o.v[0] = c0;
  o.v[1] = c1;
  o.v[2] = c2;
  o.v[3] = c3;
  return o;
}

// Draw stream for one (seed, slot, generation, tag): 32-bit draw d is half
// (d & 1) of 64-bit word (d >> 1) & 3 of block d >> 3.  Caches one block.
struct DrawStream {
  uint64_t seed, slot, gen, tag;
  uint64_t cached_block;
  Philox4x64 blk;
  __device__ DrawStream(uint64_t seed_, uint64_t slot_, uint64_t gen_, uint64_t tag_)
      : seed(seed_), slot(slot_), gen(gen_), tag(tag_), cached_block(~0ULL) {}
  __device__ __forceinline__ uint32_t draw(uint32_t d) {
    const uint64_t b = d >> 3;
    if (b != cached_block) {
      blk = philox4x64_10(b, slot, gen, tag, seed, 0);
      cached_block = b;
    }
    const uint32_t i = (d >> 1) & 3u;
    const uint64_t w = i == 0 ? blk.v[0] : i == 1 ? blk.v[1] : i == 2 ? blk.v[2] : blk.v[3];
    return (d & 1u) ? (uint32_t)(w >> 32) : (uint32_t)(w & 0xFFFFFFFFu);
  }
};

// Draws of a GA generation for nc consecutive child slots n0 .. n0+nc-1:
// DR[c*nblk*8 + d] = draw d of slot n0+c (the same values DrawStream gives;
// DR 16-byte aligned),
// one Philox block per thread (threads t0, t0 + tstride, ...).  Slots below
// E (elites) take no draws and are skipped.
__device__ __forceinline__ void gen_child_draws_from(uint32_t* DR, int n0, int nc, int nblk,
                                                     uint64_t seed, uint64_t gen, int E, int t0,
                                                     int tstride) {
  for (int t = t0; t < nc * nblk; t += tstride) {
    const int c = t / nblk, b = t - c * nblk;
    const int n = n0 + c;
    if (n < E) continue;
    const Philox4x64 r = philox4x64_10((uint64_t)b, (uint64_t)n, gen, kTagGa, seed, 0);
    // two 16-byte stores per block (DR is 16-byte aligned): the eight words
    // of consecutive threads are 32 bytes apart, so a quarter-warp covers all
    // banks once instead of eight stores hitting four banks each
    uint4* o = reinterpret_cast<uint4*>(DR + (size_t)c * nblk * 8 + b * 8);
    o[0] = make_uint4((uint32_t)(r.v[0] & 0xFFFFFFFFu), (uint32_t)(r.v[0] >> 32),
                      (uint32_t)(r.v[1] & 0xFFFFFFFFu), (uint32_t)(r.v[1] >> 32));
    o[1] = make_uint4((uint32_t)(r.v[2] & 0xFFFFFFFFu), (uint32_t)(r.v[2] >> 32),
                      (uint32_t)(r.v[3] & 0xFFFFFFFFu), (uint32_t)(r.v[3] >> 32));
  }
}

__device__ __forceinline__ void gen_child_draws(uint32_t* DR, int n0, int nc, int nblk,
                                                uint64_t seed, uint64_t gen, int E) {
  gen_child_draws_from(DR, n0, nc, nblk, seed, gen, E, threadIdx.x, blockDim.x);
}

// Uniform integer in [0, n) from a 32-bit draw (multiply-shift).
__device__ __forceinline__ uint32_t below(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

}  // namespace pa
