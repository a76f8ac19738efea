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
// FP32 kernels (throughput path).  A thread owns (chromosome, pilot p) and
// walks the L cells; for cell l it reads one row of a BS-minor table -- the
// gains of user inv_l(p) at all BSs, own-cell entry zeroed -- and adds the
// row into register accumulators (one per BS j).  Total shared-memory
// traffic per chromosome is L*K rows of NJ words: the L^2 K gathers that
// Eq. 5 needs, each word read once.  The table lives in shared memory for the
// whole (grid-stride) kernel.  Row stride RS makes every warp access
// bank-conflict free: lanes that read the same (l, u) row read the same
// address (broadcast) and distinct u land in distinct banks (float2 loads,
// RS/2 odd, K <= 16; scalar loads, RS odd, K <= 32).
//   k_eval_f32_pilot (K <= 16, L <= 24): one thread per (chromosome, pilot)
//     over all columns; chromosome tiles staged by bulk copies.
//   k_eval_f32 (other shapes): the columns split in two shares taken by the
//     two half-warps, chromosomes decoded from global memory.
//
// FP64 kernel (parity path).  One thread per user (j, k) of a chromosome,
// the oracle's operation order exactly: ascending-l sums, separately rounded
// products (no FMA), log2 by the atanh series, per-cell partial sums added in
// ascending j.
#include <algorithm>
#include <mutex>

#include "pa_eval_device.cuh"

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
  int obj;             // PA_OBJ_MIN_SINR: smallest SINR instead of the SE sum
};

template <int NJ, int VEC, bool FIN>
__global__ void __launch_bounds__(512) k_eval_f32(const F32Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* T = reinterpret_cast<float*>(smem);
  float* OWN = T + a.tab_floats;
  float* BN = OWN + ((a.L * a.K + 3) & ~3);
  float* PART = BN + ((a.L + 3) & ~3);
  uint8_t* INV = reinterpret_cast<uint8_t*>(PART + (((int64_t)a.NTK * (NJ / 2) + 3) & ~3));
  const int tid = threadIdx.x;
  const int L = a.L, K = a.K, NT = a.NT, NTK = a.NTK;
  const int64_t LK = (int64_t)L * K;

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
  const F32Smem sm{T, OWN, BN, L, K, a.RS, a.M, a.pc};

  // thread -> (member c, pilot p) index q = c*K + p and column share h; with
  // two shares, the lower and upper half-warps take shares 0 and 1 of the
  // same 16 q's, so each half-warp's float2 loads stay conflict-free
  constexpr int JS = PilotSplit<NJ, VEC>::JS;
  const int lane = tid & 31;
  const int h = JS == 2 ? (lane >> 4) : 0;
  const int q = JS == 2 ? ((tid >> 5) << 4) + (lane & 15) : tid;
  const int64_t tiles = (a.n + NT - 1) / NT;
  const bool active = q < NTK;
  const uint8_t* invp = INV + q;  // (l*NT + c)*K + p == l*NTK + q
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t n0 = tile * NT;
    const int nvalid = (int)((a.n - n0) < NT ? (a.n - n0) : NT);
    decode_members(a.pop + n0 * LK, LK, nvalid, NT, L, K, INV);
    __syncthreads();
    if (active)
      eval_pilot_f32<NJ, VEC, FIN, JS>(sm, invp, NTK, h, PART + q * (NJ / 2) + h * (NJ / 2 / JS),
                                       a.obj);
    __syncthreads();
    for (int c = tid >> 5; c < nvalid; c += blockDim.x >> 5) {
      const float* part = PART + c * K * (NJ / 2);
      const float f = a.obj ? member_min(part, K * (NJ / 2), lane)
                            : member_sum(part, K * (NJ / 2), lane);
      if (lane == 0) a.fit[n0 + c] = f;
    }
  }
}

// ------------------------------------------------------- FP32, K <= 16, L <= 24
// One thread per (member c, pilot p) over all NJ BS columns, so that the
// accumulators stay in registers and each table word is read by one thread.
// Per tile of NT members:
//   * the tile's chromosome bytes (contiguous, NT*L*K bytes, a multiple of 16)
//     arrive in shared memory by one bulk copy on an mbarrier, issued two
//     tiles ahead (double buffer);
//   * decode: one thread per (member, cell) row writes the row's inverse
//     transposed, INVT[(c*K + p)*NJ + l] = user of cell l holding pilot p, so
//     that thread (c, p) finds its users at consecutive bytes;
//   * accumulate: the same per-column ascending-l sums, SINR and SE steps as
//     eval_pilot_f32, so every per-(pilot, pair) SE and every fitness is bit
//     for bit the one the other FP32 kernels compute.
// Partial tiles, or a population not 16-byte aligned, are decoded straight
// from global memory instead.
constexpr int kPilotThreads = 256;

struct PilotArgs {
  const uint8_t* pop;
  int64_t n;
  float* fit;
  const float* tab;
  const float* own;
  const float* bn;
  int* err_flag;  // null: no bulk copies (decode from global memory)
  int L, K, RS, NT;
  int64_t tab_floats;
  int xbytes;     // shared bytes of one chromosome buffer
  int stall;      // testing: announce the bulk copies but never issue them
  float M, pc;
  int obj;        // PA_OBJ_MIN_SINR: smallest SINR instead of the SE sum
};

template <int NJ, bool FIN>
__global__ void __launch_bounds__(kPilotThreads, 4) k_eval_f32_pilot(const PilotArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_timeout;
  constexpr int NPAIR = NJ / 2;
  const int L = a.L, K = a.K, NT = a.NT, NTK = NT * K, LK = L * K;
  float* T = reinterpret_cast<float*>(smem);
  float* OWN = T + a.tab_floats;
  float* BN = OWN + ((LK + 3) & ~3);
  float* PART = BN + ((L + 3) & ~3);
  uint8_t* INVT = reinterpret_cast<uint8_t*>(PART + (((int64_t)NTK * NPAIR + 3) & ~3));
  uint8_t* X0 = INVT + ((NTK * NJ + 15) & ~15);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tiles = (a.n + NT - 1) / NT;
  const uint32_t tile_bytes = (uint32_t)NT * (uint32_t)LK;
  const bool bulk = a.err_flag != nullptr && (reinterpret_cast<uintptr_t>(a.pop) & 15) == 0 &&
                    (tile_bytes & 15) == 0;
  auto full = [&](int64_t tile) { return (tile + 1) * NT <= a.n; };
  const uint32_t mb0 = smem_u32(&mbar[0]);
  auto issue = [&](int64_t tile, int buf) {
    if (tid == 0 && bulk && tile < tiles && full(tile)) {
      const uint32_t mb = mb0 + 8 * buf;
      mbar_expect_tx(mb, tile_bytes);
      if (!a.stall)
        bulk_g2s(smem_u32(X0 + buf * a.xbytes), a.pop + tile * (int64_t)tile_bytes, tile_bytes,
                 mb);
    }
  };

  if (tid == 0) {
    mbar_init(mb0, 1);
    mbar_init(mb0 + 8, 1);
    s_timeout = 0;
  }
  {
    const float4* s4 = reinterpret_cast<const float4*>(a.tab);
    float4* d4 = reinterpret_cast<float4*>(T);
    for (int64_t i = tid; i < a.tab_floats / 4; i += blockDim.x) d4[i] = __ldg(s4 + i);
    for (int i = tid; i < LK; i += blockDim.x) OWN[i] = __ldg(a.own + i);
    if (FIN)
      for (int i = tid; i < L; i += blockDim.x) BN[i] = __ldg(a.bn + i);
    // every byte decode may skip (a pilot >= K) still names a valid user
    for (int i = tid; i < NTK * NJ / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(INVT)[i] = 0;
  }
  __syncthreads();
  issue(blockIdx.x, 0);
  issue(blockIdx.x + (int64_t)gridDim.x, 1);

  const int c_me = tid / K;
  const int KRS = K * a.RS;
  const uint8_t* inv_me = INVT + tid * NJ;
  uint32_t parity = 0;  // bit b: phase of buffer b's next completion
  int i = 0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
    const int buf = i & 1;
    const int64_t n0 = tile * NT;
    const int nvalid = (int)((a.n - n0) < NT ? (a.n - n0) : NT);
    const bool staged = bulk && full(tile);
    const uint8_t* xs = X0 + buf * a.xbytes;
    if (staged) {
      const uint32_t mb = mb0 + 8 * buf, ph = (parity >> buf) & 1;
      if (tid == 0 && !mbar_wait(mb, ph)) {
        atomicExch(a.err_flag, 1);
        // let this copy and the other buffer's (if any) land before leaving
        mbar_wait(mb, ph);
        if (tile + gridDim.x < tiles && full(tile + gridDim.x))
          mbar_wait(mb0 + 8 * (buf ^ 1), (parity >> (buf ^ 1)) & 1);
        s_timeout = 1;
      }
      __syncthreads();
      if (s_timeout) return;
      mbar_wait(mb, ph);  // complete: returns at once, orders the copied bytes
      parity ^= 1u << buf;
    }

    // ---- decode: INVT[(c*K + p)*NJ + l] = k where row (c, l) gives pilot p to
    // user k; one thread per row, cells fastest (a warp's byte stores then
    // share words or fall in distinct banks)
    for (int r = tid; r < nvalid * L; r += blockDim.x) {
      const int c = r / L, l = r - c * L;
      const int o = c * LK + l * K;
      uint8_t* dst = INVT + c * K * NJ + l;
      if (staged) {
        // the row's K <= 16 bytes, realigned from the words that hold them
        const uint32_t* w = reinterpret_cast<const uint32_t*>(xs + (o & ~3));
        const uint32_t sh = 8 * (o & 3);
        uint32_t rw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) rw[q] = __funnelshift_r(w[q], w[q + 1], sh);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t p = (rw[k >> 2] >> (8 * (k & 3))) & 0xffu;
          if (k < K && p < (uint32_t)K) dst[p * NJ] = (uint8_t)k;
        }
      } else {
        const uint8_t* row = a.pop + n0 * LK + o;
        for (int k = 0; k < K; ++k) {
          const uint32_t p = __ldg(row + k);
          if (p < (uint32_t)K) dst[p * NJ] = (uint8_t)k;
        }
      }
    }
    __syncthreads();
    issue(tile + 2 * (int64_t)gridDim.x, buf);

    // ---- accumulate over cells, then SINR / SE per BS column
    if (c_me < nvalid) {
      float2 acc2[NPAIR];
      float2 acc1[FIN ? NPAIR : 1];
#pragma unroll
      for (int q = 0; q < NPAIR; ++q) {
        acc2[q] = make_float2(0.f, 0.f);
        if (FIN) acc1[q] = make_float2(0.f, 0.f);
      }
      const float* Tl = T;
      const uint32_t* iw = reinterpret_cast<const uint32_t*>(inv_me);
      uint32_t w = 0;
#pragma unroll 4
      for (int l = 0; l < L; ++l, Tl += KRS) {
        if ((l & 3) == 0) w = iw[l >> 2];  // users of cells l .. l+3
        const int u = (w >> (8 * (l & 3))) & 0xffu;
        const float2* row = reinterpret_cast<const float2*>(Tl + u * a.RS);
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
          const float2 v = row[q];
          acc2[q] = ffma2(v, v, acc2[q]);
          if (FIN) acc1[q] = fadd2(acc1[q], v);
        }
      }
      float ps[NPAIR];
      uint32_t uw = 0;
#pragma unroll
      for (int q = 0; q < NPAIR; ++q) {
        if ((q & 1) == 0) uw = iw[q >> 1];  // users of cells 2q .. 2q+3
        const float s2[2] = {acc2[q].x, acc2[q].y};
        const float s1[2] = {FIN ? acc1[q].x : 0.f, FIN ? acc1[q].y : 0.f};
        const bool mo = a.obj != 0;
        float pse = pair_init(mo);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int j = 2 * q + hh;
          if (j < L)
            pse = pair_add(pse,
                           se_pilot_f32<FIN>(s2[hh], s1[hh],
                                             OWN[j * K + ((uw >> (8 * (j & 3))) & 0xff)],
                                             FIN ? BN[j] : 0.f, a.M, a.pc, mo),
                           mo);
        }
        ps[q] = pse;
      }
      float2* dst = reinterpret_cast<float2*>(PART + tid * NPAIR);
#pragma unroll
      for (int q = 0; q < NPAIR / 2; ++q) dst[q] = make_float2(ps[2 * q], ps[2 * q + 1]);
    }
    __syncthreads();
    float* fit = a.fit + n0;
    for (int c = warp; c < nvalid; c += kPilotThreads / 32) {
      const float f =
          member_value_bounded<16 * NPAIR>(PART + c * K * NPAIR, K * NPAIR, lane, a.obj != 0);
      if (lane == 0) fit[c] = f;
    }
  }
}

// --------------------------------------------------------------------- FP64
struct F64Args {
  const uint8_t* pop;
  int64_t n;
  double* fit;
  const double* beta;
  const double* bnc;
  int L, K;
  int fin;
  double M, pc;
  int obj;  // PA_OBJ_MIN_SINR: smallest SINR instead of the SE sum
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
      SE[r] = value_user_f64(a.beta, a.bnc, INV, L, K, j, k, X[r], a.fin, a.M, a.pc, a.obj, K, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) a.fit[n] = member_value_f64(SE, L, K, a.obj);
  }
}

// --------------------------------------------------------------------- dispatch
struct F32Launch {
  int NT, threads;
  size_t smem;
};

// Block shape of k_eval_f32: NT members of K pilots, one thread per (member,
// pilot) and column share (two shares for float2 tables with NJ >= 8).
F32Launch f32_shape(int L, int K, int RS, int NJ) {
  F32Launch s{};
  const int JS = (K <= 16 && NJ >= 8) ? 2 : 1;
  int NTK;
  if (JS == 2) {
    // up to 128 (member, pilot) pairs; 16 pairs per warp (one per column share)
    s.NT = std::max(1, 128 / K);
    NTK = s.NT * K;
    s.threads = 32 * ((NTK + 15) / 16);
  } else {
    s.NT = std::max(1, 256 / K);
    NTK = s.NT * K;
    s.threads = ((NTK + 31) / 32) * 32;
  }
  const size_t LK = (size_t)L * K;
  const size_t tab = ((LK * RS + 3) / 4) * 4;
  s.smem = 4 * (tab + ((LK + 3) & ~size_t(3)) + ((L + 3) & ~3) +
                ((size_t)NTK * (NJ / 2) + 3) / 4 * 4) +
           (((size_t)L * NTK + 15) & ~size_t(15));
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

// Block shape of k_eval_f32_pilot: NT members (NT*L*K a multiple of 16 so
// that a full tile is one bulk copy), one thread per (member, pilot).
struct PilotLaunch {
  int NT, xbytes;
  size_t smem;
};
PilotLaunch pilot_shape(int L, int K, int RS, int NJ) {
  PilotLaunch s{};
  const int LK = L * K;
  int g = 16;
  while (LK % g) g >>= 1;
  const int m = 16 / g;
  s.NT = std::max(m, (kPilotThreads / K) / m * m);
  s.xbytes = (s.NT * LK + 20 + 15) & ~15;  // +20: a row reads up to 5 words from its first
  const size_t tab = (((size_t)LK * RS + 3) / 4) * 4;
  const size_t NTK = (size_t)s.NT * K;
  s.smem = 4 * (tab + ((LK + 3) & ~size_t(3)) + ((L + 3) & ~3) + ((NTK * (NJ / 2) + 3) & ~size_t(3))) +
           ((NTK * NJ + 15) & ~size_t(15)) + 2 * (size_t)s.xbytes;
  return s;
}

bool pilot_kernel_applies(int NJ, int vec, int K) { return vec == 2 && NJ <= 24 && K <= 16; }

template <int NJ, bool FIN>
cudaError_t run_pilot(const PilotArgs& a, const PilotLaunch& s, int num_sms, cudaStream_t st) {
  auto kern = k_eval_f32_pilot<NJ, FIN>;
  cudaError_t e = cudaSuccess;
  const int per_sm = cached_occupancy((const void*)kern, kPilotThreads, s.smem, &e);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (a.n + a.NT - 1) / a.NT;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * num_sms);
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  kern<<<(unsigned)grid, kPilotThreads, s.smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <bool FIN>
cudaError_t pick_pilot(int NJ, const PilotArgs& a, const PilotLaunch& s, int sms, cudaStream_t st) {
  switch (NJ) {
    case 4: return run_pilot<4, FIN>(a, s, sms, st);
    case 8: return run_pilot<8, FIN>(a, s, sms, st);
    case 12: return run_pilot<12, FIN>(a, s, sms, st);
    case 16: return run_pilot<16, FIN>(a, s, sms, st);
    case 20: return run_pilot<20, FIN>(a, s, sms, st);
    case 24: return run_pilot<24, FIN>(a, s, sms, st);
    default: return cudaErrorInvalidValue;
  }
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
  const size_t smem = pilot_kernel_applies(NJ, vec, K) ? pilot_shape(L, K, RS, NJ).smem
                                                       : f32_shape(L, K, RS, NJ).smem;
  if (smem_bytes) *smem_bytes = smem;
  return smem <= (size_t)kSmemBudget;
}

cudaError_t launch_eval_f32(pa_ctx* ctx, const uint8_t* pop, int64_t n, float* fit,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const pa::F32Tables& t = ctx->t32;
  const int L = ctx->cfg.L, K = ctx->cfg.K;
  const bool fin = ctx->cfg.mode == PA_SINR_FINITE_M;
  if (pilot_kernel_applies(t.NJ, t.vec, K)) {
    const PilotLaunch s = pilot_shape(L, K, t.RS, t.NJ);
    PilotArgs a;
    a.pop = pop;
    a.n = n;
    a.fit = fit;
    a.tab = t.tab;
    a.own = t.own;
    a.bn = t.bn;
    a.err_flag = t.err_flag;
    a.L = L;
    a.K = K;
    a.RS = t.RS;
    a.NT = s.NT;
    a.tab_floats = (((int64_t)L * K * t.RS + 3) / 4) * 4;
    a.xbytes = s.xbytes;
    a.stall = ctx->test_stall;
    ctx->test_stall = 0;
    a.M = t.M;
    a.pc = t.pc;
    a.obj = ctx->cfg.objective;
    return fin ? pick_pilot<true>(t.NJ, a, s, ctx->num_sms, st)
               : pick_pilot<false>(t.NJ, a, s, ctx->num_sms, st);
  }
  const F32Launch s = f32_shape(L, K, t.RS, t.NJ);
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
  a.obj = ctx->cfg.objective;
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
  a.obj = ctx->cfg.objective;
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
