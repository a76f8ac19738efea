// pa_stream.cu -- population fitness (Sec. 3.2, Eq. 3-6) for instances whose
// FP32 gain table does not fit in shared memory (e.g. 61 cells x 32 users:
// 476 KB).
//
// The BS-minor table is split into tiles of JT BS columns; tile t holds, for
// every user (l, u), its gains at BSs t*JT .. t*JT+JT-1 (own-cell entries
// zero).  Each block owns one tile: it stages the tile into shared memory
// once with TMA bulk copies (cp.async.bulk completing on an mbarrier), then
// streams member tiles: decode, accumulate the per-pilot interference of the
// tile's BSs over all cells, SINR and SE for the tile's users, and a fixed-
// order per-member sum written as partial[member][tile].  A second kernel adds
// the tile partials of each member in tile order.  Waits are bounded: a copy
// that has not landed within about a second sets ctx's error flag and the
// block returns (pa_eval_population_host then reports PA_ETIMEOUT).
#include <algorithm>
#include <atomic>

#include "pa_eval_device.cuh"

namespace pa {
namespace {

struct StreamArgs {
  const uint8_t* pop;
  int64_t n;
  float* partial;  // [n][ntile]
  const float* tab;
  const float* own;
  const float* bn;
  int* err_flag;
  int L, K, RSt, ntile, NTM;
  int64_t tile_floats;
  float M, pc;
  int obj;  // PA_OBJ_MIN_SINR: smallest SINR instead of the SE sum
};

constexpr int kStreamThreads = 512;
// MINOBJ: the max-min objective (compiled apart, so the sum objective's
// inner loop carries no objective test).
template <int JT, int VEC, bool FIN, bool MINOBJ>
__global__ void __launch_bounds__(kStreamThreads) k_eval_f32_stream(const StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int s_timeout;
  const int L = a.L, K = a.K, LK = L * K, NTM = a.NTM, NTK = NTM * K, KP = inv_pitch(K);
  constexpr int NPR = JT / 2;
  float* TT = reinterpret_cast<float*>(smem);
  float* OWN = TT + a.tile_floats;
  float* BN = OWN + ((LK + 3) & ~3);
  float* PART = BN + ((L + 3) & ~3);
  uint8_t* INV = reinterpret_cast<uint8_t*>(PART + (((int64_t)NTK * NPR + 3) & ~3));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = blockIdx.x % a.ntile;
  const int b = blockIdx.x / a.ntile, nb = gridDim.x / a.ntile;

  // ---- stage tile t with bulk copies (one thread issues, all wait)
  const uint32_t mb = smem_u32(&mbar);
  if (tid == 0) {
    mbar_init(mb, 1);
    s_timeout = 0;
  }
  __syncthreads();
  const uint32_t bytes = (uint32_t)(a.tile_floats * 4);
  if (tid == 0) {
    mbar_expect_tx(mb, bytes);
    const char* src = reinterpret_cast<const char*>(a.tab + (int64_t)t * a.tile_floats);
    const uint32_t dst = smem_u32(TT);
    constexpr uint32_t kChunk = 32768;
    for (uint32_t off = 0; off < bytes; off += kChunk) {
      const uint32_t sz = bytes - off < kChunk ? bytes - off : kChunk;
      bulk_g2s(dst + off, src + off, sz, mb);
    }
  }
  for (int i = tid; i < LK; i += blockDim.x) OWN[i] = __ldg(a.own + i);
  if (FIN)
    for (int i = tid; i < L; i += blockDim.x) BN[i] = __ldg(a.bn + i);
  for (int i = tid; i < L * NTM * KP; i += blockDim.x) INV[i] = 0;
  // one thread waits (bounded) and the block leaves together on a timeout
  if (tid == 0 && !mbar_wait(mb, 0)) {
    atomicExch(a.err_flag, 1);
    mbar_wait(mb, 0);  // give the copy another bounded chance to land before leaving
    s_timeout = 1;
  }
  __syncthreads();
  if (s_timeout) return;
  mbar_wait(mb, 0);  // phase complete: returns at once, orders the copied data
  F32Smem sm{TT, OWN, BN, L, K, a.RSt, a.M, a.pc};
  sm.jbase = t * JT;

  const int64_t mtiles = (a.n + NTM - 1) / NTM;
  for (int64_t mt = b; mt < mtiles; mt += nb) {
    const int64_t n0 = mt * NTM;
    const int nvalid = (int)((a.n - n0) < NTM ? (a.n - n0) : NTM);
    decode_members_kp(a.pop + n0 * LK, LK, nvalid, NTM, L, K, KP, INV);
    __syncthreads();
    if (tid < NTK) {
      const int c = tid / K, p = tid - c * K;
      eval_pilot_f32<JT, VEC, FIN, 1>(sm, INV + c * KP + p, NTM * KP, 0, PART + tid * NPR,
                                      MINOBJ);
    }
    __syncthreads();
    for (int c = warp; c < nvalid; c += blockDim.x >> 5) {
      const float f =
          member_value_bounded<32 * NPR>(PART + c * K * NPR, K * NPR, lane, MINOBJ);
      if (lane == 0) a.partial[(n0 + c) * a.ntile + t] = f;
    }
    __syncthreads();
  }
}

// fitness[n] = sum over tiles of partial[n][t], in tile order (the smallest
// partial for the max-min objective).
__global__ void k_stream_reduce(const float* __restrict__ partial, int ntile, int64_t n,
                                float* __restrict__ fit, int minobj) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = minobj ? __int_as_float(0x7f800000) : 0.f;
    for (int t = 0; t < ntile; ++t) s = minobj ? fminf(s, partial[i * ntile + t]) : s + partial[i * ntile + t];
    fit[i] = s;
  }
}

size_t stream_smem(int L, int K, int JT, int RSt, int NTM) {
  const size_t LK = (size_t)L * K;
  const size_t tile = ((LK * RSt + 3) / 4) * 4;
  const size_t NTK = (size_t)NTM * K;
  return 4 * (tile + ((LK + 3) & ~size_t(3)) + ((L + 3) & ~3) + ((NTK * (JT / 2) + 3) & ~size_t(3))) +
         (((size_t)L * NTM * inv_pitch(K) + 15) & ~size_t(15));
}

template <int JT, int VEC, bool FIN, bool MINOBJ>
cudaError_t run_stream_obj(const StreamArgs& a, size_t smem, int grid, cudaStream_t st) {
  auto kern = k_eval_f32_stream<JT, VEC, FIN, MINOBJ>;
  static std::atomic<uint64_t> prepared{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ULL << (dev & 63);
  if (!(prepared.load() & bit)) {
    e = raise_smem_cap((const void*)kern, dev);
    if (e != cudaSuccess) return e;
    prepared.fetch_or(bit);
  }
  (void)cudaGetLastError();  // drop a stale error of an earlier call
  kern<<<grid, kStreamThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int JT, int VEC, bool FIN>
cudaError_t run_stream(const StreamArgs& a, size_t smem, int grid, cudaStream_t st) {
  return a.obj ? run_stream_obj<JT, VEC, FIN, true>(a, smem, grid, st)
               : run_stream_obj<JT, VEC, FIN, false>(a, smem, grid, st);
}

}  // namespace

// Tile geometry: the widest JT (16, else 8, else 4) whose tile, member
// buffers and partial sums fit in one CTA's shared memory.
bool f32_stream_geometry(int L, int K, int* JT, int* RSt, int* vec, int* ntile) {
  const int NTM = std::max(1, kStreamThreads / K);
  for (int jt : {16, 8, 4}) {
    const int v = K <= 16 ? 2 : 1;
    const int rs = v == 2 ? jt + 2 : jt + 1;  // RS/2 odd for float2, RS odd for scalars
    if (stream_smem(L, K, jt, rs, NTM) + 64 <= (size_t)kSmemBudget) {
      *JT = jt;
      *RSt = rs;
      *vec = v;
      *ntile = (L + jt - 1) / jt;
      return true;
    }
  }
  return false;
}

cudaError_t launch_eval_f32_stream(pa_ctx* ctx, const uint8_t* pop, int64_t n, float* fit,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pa::F32Tables& t = ctx->t32;
  if (t.partial_cap < n) {
    cudaFree(t.partial);
    t.partial = nullptr;
    t.partial_cap = 0;
    cudaError_t e = cudaMalloc(&t.partial, sizeof(float) * (size_t)n * t.ntile);
    if (e != cudaSuccess) return e;
    t.partial_cap = n;
  }
  const int L = ctx->cfg.L, K = ctx->cfg.K;
  StreamArgs a;
  a.pop = pop;
  a.n = n;
  a.partial = t.partial;
  a.tab = t.tab;
  a.own = t.own;
  a.bn = t.bn;
  a.err_flag = t.err_flag;
  a.L = L;
  a.K = K;
  a.RSt = t.RSt;
  a.ntile = t.ntile;
  a.NTM = std::max(1, kStreamThreads / K);
  a.tile_floats = t.tile_floats;
  a.M = t.M;
  a.pc = t.pc;
  a.obj = ctx->cfg.objective;
  const size_t smem = stream_smem(L, K, t.JT, t.RSt, a.NTM);
  // one block per SM (the tile fills shared memory), spread over the tiles
  const int64_t mtiles = (n + a.NTM - 1) / a.NTM;
  const int64_t want = (ctx->num_sms + t.ntile - 1) / t.ntile;
  const int per_tile = (int)std::max<int64_t>(1, std::min<int64_t>(mtiles, want));
  const int grid = per_tile * t.ntile;
  const bool fin = ctx->cfg.mode == PA_SINR_FINITE_M;
  cudaError_t e;
  if (t.vec == 2) {
    switch (t.JT) {
      case 16: e = fin ? run_stream<16, 2, true>(a, smem, grid, st) : run_stream<16, 2, false>(a, smem, grid, st); break;
      case 8: e = fin ? run_stream<8, 2, true>(a, smem, grid, st) : run_stream<8, 2, false>(a, smem, grid, st); break;
      default: e = fin ? run_stream<4, 2, true>(a, smem, grid, st) : run_stream<4, 2, false>(a, smem, grid, st); break;
    }
  } else {
    switch (t.JT) {
      case 16: e = fin ? run_stream<16, 1, true>(a, smem, grid, st) : run_stream<16, 1, false>(a, smem, grid, st); break;
      case 8: e = fin ? run_stream<8, 1, true>(a, smem, grid, st) : run_stream<8, 1, false>(a, smem, grid, st); break;
      default: e = fin ? run_stream<4, 1, true>(a, smem, grid, st) : run_stream<4, 1, false>(a, smem, grid, st); break;
    }
  }
  if (e != cudaSuccess) return e;
  const int64_t rb = std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
  (void)cudaGetLastError();
  k_stream_reduce<<<(unsigned)rb, 256, 0, st>>>(t.partial, t.ntile, n, fit, a.obj);
  count_launch();
  return cudaGetLastError();
}

}  // namespace pa
