// pa_fitness.cu -- population-wide fitness evaluation (paper Sec. 3.2).
//
// For chromosome X (row l = permutation of the K pilots over cell l's users)
// and every BS j, pilot p, the users sharing p are u_l = inv_l(p) in each
// cell l (pilots are reused across cells).  Eq. 4-5 need, per (j, p),
//   S2[j][p] = sum_{l != j} beta[j][l][u_l]^2          (coherent, pilot contamination)
// and the finite-M reading of Eq. 3 also
//   S1[j][p] = sum_l beta[j][l][u_l]                   (estimation quality)
// after which the user k = u_j of cell j has
//   sinr = b^2 / S2                                    (Eq. 4)
//   sinr = M b^2 / (M S2 + (B_j + s2/rho)(S1 + s2/(tau_p rho)))   (Eq. 3 reading)
// with b = beta[j][j][k], SE = log2(1 + sinr) (Eq. 5), fitness = sum SE (Eq. 6).
//
// FP32 kernel (throughput path).  One thread per (chromosome, pilot p).  It
// walks the L cells; for cell l it reads one row of a BS-minor table --
// the gains of user inv_l(p) at all BSs, own-cell entry zeroed -- and adds the
// row into NJ register accumulators (one per BS j).  Total shared-memory
// traffic per chromosome is L*K rows of NJ words: the L^2 K gathers that
// Eq. 5 needs, each word read once.  The table lives in shared memory for the
// whole (grid-stride) kernel.  Row stride RS makes every warp access
// bank-conflict free: lanes that read the same (l, u) row read the same
// address (broadcast) and distinct u land in distinct banks (float2 loads,
// RS/2 odd, K <= 16; scalar loads, RS odd, K <= 32).
//
// FP64 kernel (parity path).  One thread per user (j, k) of a chromosome,
// the oracle's operation order exactly: ascending-l sums, separately rounded
// products (no FMA), log2 by the atanh series, per-cell partial sums added in
// ascending j.
#include <algorithm>
#include <mutex>

#include "pa_internal.cuh"

namespace pa {
namespace {

struct F32Args {
  const uint8_t* pop;
  int64_t n;
  float* fit;
  const float* tab;
  const float* own;
  const float* bn;
  int L, K, RS, NT, NTK;
  int64_t tab_floats;  // padded to a multiple of 4
  float M, pc;
};

// Decode the pilots of NT chromosomes starting at n0 into
// inv[(l*NT + c)*K + p] = user of cell l holding pilot p in chromosome c.
// Out-of-range pilots are skipped (entries stay in range: the buffer is
// zeroed at kernel start and only ever receives values < K).
__device__ __forceinline__ void decode_tile(const F32Args& a, int64_t n0, uint8_t* inv) {
  const int L = a.L, K = a.K, NT = a.NT;
  const int64_t LK = (int64_t)L * K;
  for (int idx = threadIdx.x; idx < NT * L; idx += blockDim.x) {
    const int c = idx / L;
    const int l = idx - c * L;
    uint8_t* dst = inv + (l * NT + c) * K;
    const int64_t n = n0 + c;
    if (n < a.n) {
      const uint8_t* row = a.pop + n * LK + (int64_t)l * K;
      for (int k = 0; k < K; ++k) {
        const int p = __ldg(row + k);
        if (p < K) dst[p] = (uint8_t)k;
      }
    } else {
      for (int k = 0; k < K; ++k) dst[k] = (uint8_t)k;
    }
  }
}

template <int NJ, int VEC, bool FIN>
__global__ void __launch_bounds__(512) k_eval_f32(const F32Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* T = reinterpret_cast<float*>(smem);
  float* OWN = T + a.tab_floats;
  float* BN = OWN + ((a.L * a.K + 3) & ~3);
  float* PART = BN + ((a.L + 3) & ~3);
  uint8_t* INV = reinterpret_cast<uint8_t*>(PART + ((a.NTK + 3) & ~3));
  const int tid = threadIdx.x;
  const int L = a.L, K = a.K, NT = a.NT, NTK = a.NTK, RS = a.RS;

  // Stage the instance tables once per block.
  {
    const float4* s4 = reinterpret_cast<const float4*>(a.tab);
    float4* d4 = reinterpret_cast<float4*>(T);
    for (int64_t i = tid; i < a.tab_floats / 4; i += blockDim.x) d4[i] = __ldg(s4 + i);
    for (int i = tid; i < L * K; i += blockDim.x) OWN[i] = __ldg(a.own + i);
    if (FIN)
      for (int i = tid; i < L; i += blockDim.x) BN[i] = __ldg(a.bn + i);
    for (int i = tid; i < L * NTK; i += blockDim.x) INV[i] = 0;
  }
  __syncthreads();

  const int64_t tiles = (a.n + NT - 1) / NT;
  const bool active = tid < NTK;
  const uint8_t* invp = INV + tid;  // (l*NT + c)*K + p == l*NTK + tid
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t n0 = tile * NT;
    decode_tile(a, n0, INV);
    __syncthreads();
    if (active) {
      float acc2[NJ];
      float acc1[FIN ? NJ : 1];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        acc2[j] = 0.f;
        if (FIN) acc1[j] = 0.f;
      }
      const float* Tl = T;
      for (int l = 0; l < L; ++l, Tl += K * RS) {
        const int u = invp[l * NTK];
        const float* row = Tl + u * RS;
        if (VEC == 2) {
          const float2* row2 = reinterpret_cast<const float2*>(row);
#pragma unroll
          for (int c = 0; c < NJ / 2; ++c) {
            const float2 t = row2[c];
            acc2[2 * c] = fmaf(t.x, t.x, acc2[2 * c]);
            acc2[2 * c + 1] = fmaf(t.y, t.y, acc2[2 * c + 1]);
            if (FIN) {
              acc1[2 * c] += t.x;
              acc1[2 * c + 1] += t.y;
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < NJ; ++c) {
            const float t = row[c];
            acc2[c] = fmaf(t, t, acc2[c]);
            if (FIN) acc1[c] += t;
          }
        }
      }
      float se = 0.f;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (j < L) {
          const int u = invp[j * NTK];
          const float b = OWN[j * K + u];
          const float b2 = b * b;
          float num, den;
          if (FIN) {
            num = a.M * b2;
            den = fmaf(a.M, acc2[j], BN[j] * (acc1[j] + b + a.pc));
          } else {
            num = b2;
            den = acc2[j];
          }
          se += __log2f(1.f + __fdividef(num, den));
        }
      }
      PART[tid] = se;
    }
    __syncthreads();
    if (tid < NT && n0 + tid < a.n) {
      float s = 0.f;
      for (int p = 0; p < K; ++p) s += PART[tid * K + p];
      a.fit[n0 + tid] = s;
    }
  }
}

// --------------------------------------------------------------------- FP64
// log2 by the atanh series ln m = 2 sum_{n>=0} s^(2n+1)/(2n+1), s = (m-1)/(m+1)
// (Abramowitz & Stegun 4.1.27) after x = m 2^e, m in [sqrt(1/2), sqrt(2));
// every operation separately rounded so that the result is reproducible.
__device__ __forceinline__ double log2_series(double x) {
  if (isinf(x)) return x;
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7ff) - 1022;  // x = f 2^E, f in [0.5, 1)
  const double f = __longlong_as_double((bits & 0x800FFFFFFFFFFFFFLL) | 0x3FE0000000000000LL);
  double m;
  int e;
  if (f < 0.70710678118654752440) {
    m = __dmul_rn(f, 2.0);
    e = E - 1;
  } else {
    m = f;
    e = E;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double t = __dmul_rn(s, s);
  double p = 1.0 / 23.0;
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 21.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 19.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 17.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 15.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 13.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 11.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 9.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 7.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 5.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0 / 3.0);
  p = __dadd_rn(__dmul_rn(p, t), 1.0);
  const double ln_m = __dmul_rn(__dmul_rn(2.0, s), p);
  return __dadd_rn((double)e, __dmul_rn(ln_m, 1.44269504088896340736));
}

struct F64Args {
  const uint8_t* pop;
  int64_t n;
  double* fit;
  const double* beta;
  const double* bnc;
  int L, K;
  int fin;
  double M, pc;
};

__global__ void __launch_bounds__(256) k_eval_f64(const F64Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.L, K = a.K, LK = L * K;
  double* SE = reinterpret_cast<double*>(smem);
  uint8_t* X = reinterpret_cast<uint8_t*>(SE + LK);
  uint8_t* INV = X + LK;
  for (int i = threadIdx.x; i < LK; i += blockDim.x) INV[i] = 0;
  for (int64_t n = blockIdx.x; n < a.n; n += gridDim.x) {
    __syncthreads();
    const uint8_t* src = a.pop + n * LK;
    for (int r = threadIdx.x; r < LK; r += blockDim.x) {
      const int l = r / K, k = r - l * K;
      int p = __ldg(src + r);
      p = p < K ? p : K - 1;
      X[r] = (uint8_t)p;
      INV[l * K + p] = (uint8_t)k;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < LK; r += blockDim.x) {
      const int j = r / K, k = r - j * K;
      const int p = X[r];
      const double* bj = a.beta + (size_t)j * LK;
      double s2 = 0.0, s1 = 0.0;
      for (int l = 0; l < L; ++l) {
        const double b = __ldg(bj + l * K + INV[l * K + p]);
        if (a.fin) s1 = __dadd_rn(s1, b);
        if (l != j) s2 = __dadd_rn(s2, __dmul_rn(b, b));
      }
      const double own = __ldg(bj + j * K + k);
      const double own2 = __dmul_rn(own, own);
      double sinr;
      if (a.fin) {
        const double num = __dmul_rn(a.M, own2);
        const double den =
            __dadd_rn(__dmul_rn(a.M, s2), __dmul_rn(__ldg(a.bnc + j), __dadd_rn(s1, a.pc)));
        sinr = __ddiv_rn(num, den);
      } else {
        sinr = __ddiv_rn(own2, s2);
      }
      SE[r] = log2_series(__dadd_rn(1.0, sinr));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double fitness = 0.0;
      for (int j = 0; j < L; ++j) {
        double cell = 0.0;
        for (int k = 0; k < K; ++k) cell = __dadd_rn(cell, SE[j * K + k]);
        fitness = __dadd_rn(fitness, cell);
      }
      a.fit[n] = fitness;
    }
  }
}

// --------------------------------------------------------------------- dispatch
struct F32Launch {
  int NT, threads;
  size_t smem;
};

F32Launch f32_shape(int L, int K, int RS) {
  F32Launch s{};
  if (K <= 16) {
    int base = 32;
    while (base % K) base += 32;  // lcm(K, 32)
    const int m = std::max(1, 256 / base);
    s.threads = base * m;
    s.NT = s.threads / K;
  } else {
    s.NT = std::max(1, 256 / K);
    s.threads = ((s.NT * K + 31) / 32) * 32;
  }
  const size_t LK = (size_t)L * K;
  const size_t tab = ((LK * RS + 3) / 4) * 4;
  const size_t NTK = (size_t)s.NT * K;
  s.smem = 4 * (tab + ((LK + 3) & ~size_t(3)) + ((L + 3) & ~3) + ((NTK + 3) & ~size_t(3))) +
           ((L * NTK + 15) & ~size_t(15));
  return s;
}

// Resident blocks per SM of a kernel at a launch shape.  The first query of
// a kernel on a device raises its dynamic shared-memory cap to the device's
// opt-in maximum (a cap sized to one launch would reject a later, larger
// one); the queries cost host time, so results are cached per (kernel,
// device, threads, shared memory).
struct OccKey {
  const void* fn;
  int dev, threads;
  size_t smem;
};
static int cached_occupancy(const void* fn, int threads, size_t smem, cudaError_t* err) {
  static OccKey keys[256];
  static int vals[256];
  static int used = 0;
  static const void* capped_fn[64];
  static int capped_dev[64];
  static int ncapped = 0;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return 0;
  for (int i = 0; i < used; ++i)
    if (keys[i].fn == fn && keys[i].dev == dev && keys[i].threads == threads &&
        keys[i].smem == smem)
      return vals[i];
  bool capped = false;
  for (int i = 0; i < ncapped; ++i) capped |= (capped_fn[i] == fn && capped_dev[i] == dev);
  if (!capped) {
    *err = raise_smem_cap(fn, dev);
    if (*err != cudaSuccess) return 0;
    if (ncapped < 64) {
      capped_fn[ncapped] = fn;
      capped_dev[ncapped] = dev;
      ++ncapped;
    }
  }
  int per_sm = 0;
  *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (*err != cudaSuccess) return 0;
  if (used < 256) {
    keys[used] = OccKey{fn, dev, threads, smem};
    vals[used] = per_sm;
    ++used;
  }
  return per_sm;
}

template <int NJ, int VEC, bool FIN>
cudaError_t run_f32(const F32Args& a, const F32Launch& s, int num_sms, cudaStream_t st) {
  auto kern = k_eval_f32<NJ, VEC, FIN>;
  cudaError_t e = cudaSuccess;
  const int per_sm = cached_occupancy((const void*)kern, s.threads, s.smem, &e);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (a.n + a.NT - 1) / a.NT;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * num_sms);
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  kern<<<(unsigned)grid, s.threads, s.smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int VEC, bool FIN>
cudaError_t pick_nj(int NJ, const F32Args& a, const F32Launch& s, int sms, cudaStream_t st) {
  switch (NJ) {
    case 4: return run_f32<4, VEC, FIN>(a, s, sms, st);
    case 8: return run_f32<8, VEC, FIN>(a, s, sms, st);
    case 12: return run_f32<12, VEC, FIN>(a, s, sms, st);
    case 16: return run_f32<16, VEC, FIN>(a, s, sms, st);
    case 20: return run_f32<20, VEC, FIN>(a, s, sms, st);
    case 24: return run_f32<24, VEC, FIN>(a, s, sms, st);
    case 28: return run_f32<28, VEC, FIN>(a, s, sms, st);
    case 32: return run_f32<32, VEC, FIN>(a, s, sms, st);
    case 36: return run_f32<36, VEC, FIN>(a, s, sms, st);
    case 40: return run_f32<40, VEC, FIN>(a, s, sms, st);
    case 44: return run_f32<44, VEC, FIN>(a, s, sms, st);
    case 48: return run_f32<48, VEC, FIN>(a, s, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Row geometry of the FP32 table for an (L, K) instance.
void f32_geometry(int L, int K, int* NJ, int* RS, int* vec) {
  *NJ = std::max(4, ((L + 3) / 4) * 4);
  *vec = K <= 16 ? 2 : 1;
  *RS = (*vec == 2) ? *NJ + 2 : *NJ + 1;  // RS/2 odd, or RS odd
}

bool f32_supported(int L, int K, size_t* smem_bytes) {
  int NJ, RS, vec;
  f32_geometry(L, K, &NJ, &RS, &vec);
  if (NJ > kMaxNJ || K > kMaxK) return false;
  const F32Launch s = f32_shape(L, K, RS);
  if (smem_bytes) *smem_bytes = s.smem;
  return s.smem <= (size_t)kSmemBudget;
}

cudaError_t launch_eval_f32(const pa_ctx* ctx, const uint8_t* pop, int64_t n, float* fit,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const pa::F32Tables& t = ctx->t32;
  const int L = ctx->cfg.L, K = ctx->cfg.K;
  const F32Launch s = f32_shape(L, K, t.RS);
  F32Args a;
  a.pop = pop;
  a.n = n;
  a.fit = fit;
  a.tab = t.tab;
  a.own = t.own;
  a.bn = t.bn;
  a.L = L;
  a.K = K;
  a.RS = t.RS;
  a.NT = s.NT;
  a.NTK = s.NT * K;
  a.tab_floats = (((int64_t)L * K * t.RS + 3) / 4) * 4;
  a.M = t.M;
  a.pc = t.pc;
  const bool fin = ctx->cfg.mode == PA_SINR_FINITE_M;
  if (t.vec == 2)
    return fin ? pick_nj<2, true>(t.NJ, a, s, ctx->num_sms, st)
               : pick_nj<2, false>(t.NJ, a, s, ctx->num_sms, st);
  return fin ? pick_nj<1, true>(t.NJ, a, s, ctx->num_sms, st)
             : pick_nj<1, false>(t.NJ, a, s, ctx->num_sms, st);
}

cudaError_t launch_eval_f64(const pa_ctx* ctx, const uint8_t* pop, int64_t n, double* fit,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  F64Args a;
  a.pop = pop;
  a.n = n;
  a.fit = fit;
  a.beta = ctx->beta64;
  a.bnc = ctx->bnc64;
  a.L = ctx->cfg.L;
  a.K = ctx->cfg.K;
  a.fin = ctx->cfg.mode == PA_SINR_FINITE_M;
  a.M = ctx->cfg.M;
  a.pc = ctx->pc;
  const int LK = a.L * a.K;
  const size_t smem = (size_t)LK * 8 + 2 * (size_t)LK;
  const int threads = LK >= 256 ? 256 : ((LK + 31) / 32) * 32;
  cudaError_t e = cudaSuccess;
  cached_occupancy((const void*)k_eval_f64, threads, smem, &e);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(n, (int64_t)ctx->num_sms * 8);
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  k_eval_f64<<<(unsigned)grid, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace pa
