// pa_eval_device.cuh -- device-side pieces of the fitness evaluation
// (paper Sec. 3.2, Eq. 3-6) shared by the population kernels of
// pa_fitness.cu and the fused solve kernel of pa_solve.cu.
#pragma once

#include "pa_internal.cuh"

namespace pa {

// ----------------------------------------------------------------- async copies
// Bulk global->shared copies completing on an mbarrier (TMA engine), and a
// bounded wait on the barrier's phase.
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
               : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mb) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(mb)
      : "memory");
}
// Wait for phase `parity` of an mbarrier; false after about a second.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// ----------------------------------------------------------------- decode
// Pilot -> user maps of NT members: INV[(l*NT + c)*K + p] = k where member c
// gives pilot p to user k of cell l.  Member c's row l starts at
// src + c*member_stride + l*K (generic pointer: global or shared memory).
// Members c >= nvalid get the identity.  Consecutive threads take
// consecutive members of one cell, so their K-byte targets are adjacent.
// Out-of-range pilots are skipped: INV only ever holds values < K provided
// it was initialised (e.g. zeroed) once.
__device__ __forceinline__ void decode_members(const uint8_t* src, int64_t member_stride,
                                               int nvalid, int NT, int L, int K,
                                               uint8_t* INV) {
  for (int idx = threadIdx.x; idx < NT * L; idx += blockDim.x) {
    const int l = idx / NT;
    const int c = idx - l * NT;
    uint8_t* dst = INV + idx * K;
    if (c < nvalid) {
      const uint8_t* row = src + c * member_stride + (int64_t)l * K;
      for (int k = 0; k < K; ++k) {
        const int p = row[k];
        if (p < K) dst[p] = (uint8_t)k;
      }
    } else {
      for (int k = 0; k < K; ++k) dst[k] = (uint8_t)k;
    }
  }
}

// Same as decode_members with a row pitch KP >= K (KP/4 odd keeps the rows
// of consecutive members in distinct banks): INV[(l*NT + c)*KP + p] = k.
// Rows are read with 16- or 4-byte loads when K and the addresses allow.
__device__ __forceinline__ void decode_members_kp(const uint8_t* src, int64_t member_stride,
                                                  int nvalid, int NT, int L, int K, int KP,
                                                  uint8_t* INV) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(src);
  const bool v16 = K % 16 == 0 && base % 16 == 0 && member_stride % 16 == 0;
  const bool v4 = !v16 && K % 4 == 0 && base % 4 == 0 && member_stride % 4 == 0;
  for (int idx = threadIdx.x; idx < NT * L; idx += blockDim.x) {
    const int l = idx / NT;
    const int c = idx - l * NT;
    uint8_t* dst = INV + idx * KP;
    if (c < nvalid) {
      const uint8_t* row = src + c * member_stride + (int64_t)l * K;
      if (v16) {
        for (int k0 = 0; k0 < K; k0 += 16) {
          const uint4 w = __ldg(reinterpret_cast<const uint4*>(row + k0));
          const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int p = (ws[j >> 2] >> (8 * (j & 3))) & 0xff;
            if (p < K) dst[p] = (uint8_t)(k0 + j);
          }
        }
      } else if (v4) {
        for (int k0 = 0; k0 < K; k0 += 4) {
          const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(row + k0));
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int p = (w >> (8 * j)) & 0xff;
            if (p < K) dst[p] = (uint8_t)(k0 + j);
          }
        }
      } else {
        for (int k = 0; k < K; ++k) {
          const int p = row[k];
          if (p < K) dst[p] = (uint8_t)k;
        }
      }
    } else {
      for (int k = 0; k < K; ++k) dst[k] = (uint8_t)k;
    }
  }
}

// Row pitch for decode_members_kp: K rounded up to 4 bytes, an odd number
// of words.
__host__ __device__ __forceinline__ int inv_pitch(int K) {
  int kp = (K + 3) & ~3;
  if ((kp / 4) % 2 == 0) kp += 4;
  return kp;
}

// ----------------------------------------------------------------- FP32
// Packed two-lane FP32 arithmetic (sm_100 f32x2 instructions): one
// instruction, two independent IEEE single-precision operations, each
// rounded exactly as the scalar one.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Read-only view of the FP32 tables staged in shared memory.
struct F32Smem {
  const float* T;    // [L*K rows][RS], own-cell entry zero
  const float* OWN;  // [L*K]
  const float* BN;   // [L]
  int L, K, RS;
  float M, pc;
  int jbase = 0;     // BS index of the table's first column (column tiles)
};

// Hardware approximations (MUFU) with subnormals flushed: the arguments here
// are normal numbers (gains are scaled to at most 1; sums of squares of them
// stay far above 2^-126), so flushing costs nothing and saves the fix-up
// instructions of the non-flushing forms.
__device__ __forceinline__ float rcp_ftz(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_ftz(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Objective value of one user from its pilot's sums at its own BS j (Eq.
// 4-5, or the finite-M reading of Eq. 3): s2 = sum_{l != j} of squared gains,
// s1 = sum over l != j of gains, b = own gain, bn = B_j + s2/rho (scaled).
// minobj false: SE = log2(1 + SINR) (Eq. 5, summed by the sum-SE objective
// of Eq. 7); true: the SINR itself (the max-min objective of Sec. 2).  Every
// FP32 kernel takes this exact sequence of roundings (the intrinsics fix
// where a multiply-add is fused).
template <bool FIN>
__device__ __forceinline__ float se_pilot_f32(float s2, float s1, float b, float bn, float M,
                                              float pc, bool minobj) {
  const float b2 = b * b;
  float num, den;
  if (FIN) {
    num = M * b2;
    den = fmaf(M, s2, bn * (s1 + b + pc));
  } else {
    num = b2;
    den = s2;
  }
  const float r = rcp_ftz(den);
  return minobj ? __fmul_rn(num, r) : lg2_ftz(__fmaf_rn(num, r, 1.f));
}

// Combine two users' values of one (pilot, column pair) entry: a sum for the
// sum-SE objective (starting from 0), a minimum for the max-min objective
// (starting from +inf, so that padding columns leave the entry unchanged).
__device__ __forceinline__ float pair_init(bool minobj) { return minobj ? __int_as_float(0x7f800000) : 0.f; }
__device__ __forceinline__ float pair_add(float acc, float v, bool minobj) {
  return minobj ? fminf(acc, v) : acc + v;
}

// Threads per (member, pilot) of the batch FP32 evaluation: two for float2
// tables with at least 8 BS columns (each takes half of the columns), else one.
template <int NJ, int VEC>
struct PilotSplit {
  static constexpr int JS = (VEC == 2 && NJ >= 8) ? 2 : 1;
};

// SE of the users holding pilot p in one member, for the BS column pairs
// [h*NP, (h+1)*NP) with NP = NJ/(2 JS); invp[l*stride] is the user of cell l
// holding p.  For each cell l the row of user inv_l(p) (its gains at every
// BS) is added into the accumulators, squared for S2 and plain for S1
// (FINITE_M).  pair_se[c] receives se(2c) + se(2c+1) for each pair c of the
// share (zero for columns past L), so that the member's fitness can be
// summed over (pilot, pair) in one fixed order whatever JS is.
template <int NJ, int VEC, bool FIN, int JS>
__device__ __forceinline__ void eval_pilot_f32(const F32Smem& s, const uint8_t* invp, int stride,
                                               int h, float* pair_se, bool minobj) {
  static_assert(NJ % (2 * JS) == 0, "NJ must split into JS shares of column pairs");
  constexpr int NP = NJ / 2 / JS;
  float2 acc2[NP];
  float2 acc1[FIN ? NP : 1];
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    acc2[c] = make_float2(0.f, 0.f);
    if (FIN) acc1[c] = make_float2(0.f, 0.f);
  }
  const int L = s.L, K = s.K, RS = s.RS;
  const int c0 = h * NP;
  const float* Tl = s.T + 2 * c0;
#pragma unroll 2
  for (int l = 0; l < L; ++l) {
    const int u = invp[l * stride];
    const float* row = Tl + (l * K + u) * RS;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      float2 v;
      if (VEC == 2)
        v = reinterpret_cast<const float2*>(row)[c];
      else
        v = make_float2(row[2 * c], row[2 * c + 1]);
      acc2[c] = ffma2(v, v, acc2[c]);
      if (FIN) acc1[c] = fadd2(acc1[c], v);
    }
  }
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    const float s2[2] = {acc2[c].x, acc2[c].y};
    const float s1[2] = {FIN ? acc1[c].x : 0.f, FIN ? acc1[c].y : 0.f};
    float ps = pair_init(minobj);
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int j = s.jbase + 2 * (c0 + c) + hh;
      if (j < L) {
        const int u = invp[j * stride];
        ps = pair_add(ps, se_pilot_f32<FIN>(s2[hh], s1[hh], s.OWN[j * K + u], FIN ? s.BN[j] : 0.f,
                                            s.M, s.pc, minobj),
                      minobj);
      }
    }
    pair_se[c] = ps;
  }
}

// Fitness of one member from its n per-(pilot, pair) SE sums, by one warp:
// lane i adds entries i, i+32, ... in order, then a fixed xor-shuffle tree.
// Every kernel sums the same entries this way, so their results agree.
__device__ __forceinline__ float member_sum(const float* part, int n, int lane) {
  float s = 0.f;
  for (int i = lane; i < n; i += 32) s += part[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// member_sum with the first NMAX entries (a multiple of 32) in an unrolled
// loop: the same additions in the same order.
template <int NMAX>
__device__ __forceinline__ float member_sum_bounded(const float* part, int n, int lane) {
  static_assert(NMAX % 32 == 0, "whole rounds of 32 entries");
  float s = 0.f;
#pragma unroll
  for (int i0 = 0; i0 < NMAX; i0 += 32)
    if (i0 + lane < n) s += part[i0 + lane];
  for (int i = NMAX + lane; i < n; i += 32) s += part[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// The max-min objective's counterparts of member_sum / member_sum_bounded:
// the smallest of the member's entries (a minimum is exact in any order).
__device__ __forceinline__ float member_min(const float* part, int n, int lane) {
  float s = __int_as_float(0x7f800000);
  for (int i = lane; i < n; i += 32) s = fminf(s, part[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fminf(s, __shfl_xor_sync(0xffffffffu, s, off));
  return s;
}

template <int NMAX>
__device__ __forceinline__ float member_min_bounded(const float* part, int n, int lane) {
  static_assert(NMAX % 32 == 0, "whole rounds of 32 entries");
  float s = __int_as_float(0x7f800000);
#pragma unroll
  for (int i0 = 0; i0 < NMAX; i0 += 32)
    if (i0 + lane < n) s = fminf(s, part[i0 + lane]);
  for (int i = NMAX + lane; i < n; i += 32) s = fminf(s, part[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fminf(s, __shfl_xor_sync(0xffffffffu, s, off));
  return s;
}

// Member fitness under either objective.
template <int NMAX>
__device__ __forceinline__ float member_value_bounded(const float* part, int n, int lane,
                                                      bool minobj) {
  return minobj ? member_min_bounded<NMAX>(part, n, lane) : member_sum_bounded<NMAX>(part, n, lane);
}

// ----------------------------------------------------------------- FP64
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

// SINR of user k of cell j with pilot p in one member (FP64, the oracle's
// operation order): inv[l*ls + q*ps] = user of cell l holding pilot q (ls =
// K, ps = 1 for row-major inverse rows; ls = 1, ps = pitch for pilot-major).
__device__ __forceinline__ double sinr_user_f64(const double* __restrict__ beta,
                                                const double* __restrict__ bnc, const uint8_t* inv,
                                                int L, int K, int j, int k, int p, int fin,
                                                double M, double pc, int ls, int ps) {
  const double* bj = beta + (size_t)j * L * K;
  double s2 = 0.0, s1 = 0.0;
  for (int l = 0; l < L; ++l) {
    const double b = __ldg(bj + l * K + inv[l * ls + p * ps]);
    if (fin) s1 = __dadd_rn(s1, b);
    if (l != j) s2 = __dadd_rn(s2, __dmul_rn(b, b));
  }
  const double own = __ldg(bj + j * K + k);
  const double own2 = __dmul_rn(own, own);
  double sinr;
  if (fin) {
    const double num = __dmul_rn(M, own2);
    const double den = __dadd_rn(__dmul_rn(M, s2), __dmul_rn(__ldg(bnc + j), __dadd_rn(s1, pc)));
    sinr = __ddiv_rn(num, den);
  } else {
    sinr = __ddiv_rn(own2, s2);
  }
  return sinr;
}

// Objective value of that user: SE = log2(1 + SINR) (Eq. 5) for the sum-SE
// objective, the SINR itself for the max-min objective.
__device__ __forceinline__ double value_user_f64(const double* __restrict__ beta,
                                                 const double* __restrict__ bnc,
                                                 const uint8_t* inv, int L, int K, int j, int k,
                                                 int p, int fin, double M, double pc, int minobj,
                                                 int ls, int ps) {
  const double sinr = sinr_user_f64(beta, bnc, inv, L, K, j, k, p, fin, M, pc, ls, ps);
  return minobj ? sinr : log2_series(__dadd_rn(1.0, sinr));
}

// Eq. 6 sum of one member's per-user SE (se[j*K + k]) in the oracle's order:
// per cell over k, then over cells.
__device__ __forceinline__ double sum_se_f64(const double* se, int L, int K) {
  double fitness = 0.0;
  for (int j = 0; j < L; ++j) {
    double cell = 0.0;
    for (int k = 0; k < K; ++k) cell = __dadd_rn(cell, se[j * K + k]);
    fitness = __dadd_rn(fitness, cell);
  }
  return fitness;
}

// Member fitness from its per-user values: the Eq. 6 sum, or the smallest
// value (max-min objective).
__device__ __forceinline__ double member_value_f64(const double* v, int L, int K, int minobj) {
  if (!minobj) return sum_se_f64(v, L, K);
  double m = v[0];
  for (int i = 1; i < L * K; ++i) m = fmin(m, v[i]);
  return m;
}

}  // namespace pa
