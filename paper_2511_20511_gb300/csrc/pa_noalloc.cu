// pa_noalloc.cu -- fitness evaluation for callers that cannot allocate GPU
// memory.
//
// pa_eval_population needs a context, and pa_create allocates device memory
// for the instance (gains, prepared tables, population buffers).  Some
// callers cannot do that: a real-time scheduler loop that must never hit
// the implicit device synchronisation and unbounded latency of cudaMalloc,
// or a host framework that owns all device memory through its own pool.
// pa_eval_population_noalloc gives them the same result
// without any allocation: the instance data and the prepared tables live in
// one file-scope device array, g_noalloc_scratch, of kNoallocBytes bytes
// that every GPU holds from the moment this library is loaded until the
// process exits.
//
// Sharing rules: every call uses the same array and leaves its contents
// behind; each call rewrites every byte it later reads before reading it,
// so nothing carries over from one call to the next.  Two calls whose GPU
// work overlaps (different streams without ordering, or different host
// threads on one device) race on the array and give undefined results.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pa_internal.cuh"

namespace pa {

void f32_geometry(int L, int K, int* NJ, int* RS, int* vec);
bool config_ok(const pa_config* c, std::string* why);
void set_thread_error(const std::string& msg);

constexpr size_t kNoallocBytes = PA_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol names a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
static cudaError_t scratch_address(int dev, unsigned char** out) {
  static unsigned char* addr[64] = {};
  static std::mutex mu;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = addr[dev];
  return cudaSuccess;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace pa

extern "C" pa_status pa_eval_population_noalloc(const pa_config* cfg, const double* beta,
                                                const uint8_t* pop_dev, int64_t n, void* fit_dev,
                                                void* stream) {
  using namespace pa;
  std::string why;
  set_thread_error("");  // a failure of an earlier call must not outlive this one
  if (!cfg || !beta) {
    set_thread_error("cfg and beta are required");
    return PA_EINVAL;
  }
  if (!config_ok(cfg, &why)) {
    set_thread_error(why);
    return PA_EINVAL;
  }
  if (n < 0) {
    set_thread_error("n must be >= 0");
    return PA_EINVAL;
  }
  double bmax = 0.0;
  if (!instance_ok(*cfg, beta, nullptr, nullptr, &bmax)) {
    set_thread_error("beta must be finite and > 0");
    return PA_EINVAL;
  }
  const int L = cfg->L, K = cfg->K;
  if (cfg->prec == PA_FP32 && !f32_supported(L, K, nullptr)) {
    set_thread_error("FP32 gain table of this (L, K) exceeds shared memory");
    return PA_EUNSUPPORTED;
  }
  if (n == 0) return PA_OK;
  if (!pop_dev || !fit_dev) {
    set_thread_error("null buffer");
    return PA_EINVAL;
  }
  // Layout inside the static array: beta | bnc | FP32 table | own | bn.
  const int64_t LK = (int64_t)L * K, n_beta = LK * L;
  int NJ = 0, RS = 0, vec = 0;
  if (cfg->prec == PA_FP32) f32_geometry(L, K, &NJ, &RS, &vec);
  const int64_t tab_floats = cfg->prec == PA_FP32 ? ((LK * RS + 3) / 4) * 4 : 0;
  const size_t off_beta = 0;
  const size_t off_bnc = align256(off_beta + sizeof(double) * n_beta);
  const size_t off_tab = align256(off_bnc + sizeof(double) * L);
  const size_t off_own = align256(off_tab + sizeof(float) * tab_floats);
  const size_t off_bn = align256(off_own + sizeof(float) * (cfg->prec == PA_FP32 ? LK : 0));
  const size_t need = off_bn + sizeof(float) * (cfg->prec == PA_FP32 ? L : 0);
  if (need > kNoallocBytes) {
    set_thread_error("instance needs " + std::to_string(need) + " bytes of scratch; the static "
                     "array holds " + std::to_string(kNoallocBytes));
    return PA_EUNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  unsigned char* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_thread_error(std::string("scratch set-up: ") + cudaGetErrorString(e));
    return PA_ECUDA;
  }
  // A context object on the host stack pointing into the static array: the
  // regular launchers run unchanged on it.
  pa_ctx c;
  c.cfg = *cfg;
  c.device = dev;
  c.num_sms = sms;
  c.stream = static_cast<cudaStream_t>(stream);
  c.nc = cfg->sigma2 / cfg->rho;
  c.pc = cfg->sigma2 / ((double)cfg->tau_p * cfg->rho);
  c.beta64 = reinterpret_cast<double*>(base + off_beta);
  c.bnc64 = reinterpret_cast<double*>(base + off_bnc);
  if (cfg->prec == PA_FP32) {
    int e2 = 0;
    std::frexp(bmax, &e2);
    c.t32.tab = reinterpret_cast<float*>(base + off_tab);
    c.t32.own = reinterpret_cast<float*>(base + off_own);
    c.t32.bn = reinterpret_cast<float*>(base + off_bn);
    c.t32.NJ = NJ;
    c.t32.RS = RS;
    c.t32.vec = vec;
    c.t32.scale_exp = -e2;
    c.t32.scale = std::ldexp(1.0, -e2);
    c.t32.M = (float)cfg->M;
    c.t32.pc = (float)std::ldexp(c.pc, -e2);
  }
  e = cudaMemcpyAsync(c.beta64, beta, sizeof(double) * n_beta, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = launch_prep(&c);
  if (e == cudaSuccess)
    e = cfg->prec == PA_FP64
            ? launch_eval_f64(&c, pop_dev, n, static_cast<double*>(fit_dev), c.stream)
            : launch_eval_f32(&c, pop_dev, n, static_cast<float*>(fit_dev), c.stream);
  // the beta copy may still be reading the caller's host array
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    set_thread_error(std::string("noalloc eval: ") + cudaGetErrorString(e));
    return PA_ECUDA;
  }
  return PA_OK;
}
