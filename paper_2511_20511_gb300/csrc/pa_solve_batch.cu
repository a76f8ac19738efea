// pa_solve_batch.cu -- many instances per launch: persistent thread-block
// clusters take the next instance from a counter and run the whole GA on it
// (the same device code as the one-instance kernel, pa_solve_body.cuh); the
// argument records, launch shapes and CTA sizes of the batch and server paths.
// The throughput column split is instantiated here; the latency split (the
// one-instance kernel's, for a few concurrent instances) in
// pa_solve_batch_lat.cu.
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "pa_solve_batch.cuh"

namespace pa {

cudaError_t dispatch_batch_latency(const pa_ctx* proto, int C, int clusters, const void* d, int n,
                                   int* ctr, size_t smem, bool q, int* mc, cudaStream_t st);
cudaError_t dispatch_batch_small(const pa_ctx* proto, int C, int clusters, const void* d, int n,
                                 int* ctr, size_t smem, bool q, int* mc, cudaStream_t st);

static cudaError_t dispatch_any(bool latency, int threads, const pa_ctx* proto, int C,
                                int clusters, const SolveArgs* d, int n, int* ctr, size_t smem,
                                bool q, int* mc, cudaStream_t st) {
  if (latency) return dispatch_batch_latency(proto, C, clusters, d, n, ctr, smem, q, mc, st);
  if (threads == kSmallCtaThreads)
    return dispatch_batch_small(proto, C, clusters, d, n, ctr, smem, q, mc, st);
  return dispatch_batch<kBatchMaxNP, kSolveThreads>(proto, C, clusters, d, n, ctr, smem, q, mc, st);
}

size_t solve_args_bytes() { return sizeof(SolveArgs); }

// Arguments of one instance's solve with cluster size C (written to
// args_out, a SolveArgs); returns the shared memory it needs, or 0 when it
// does not fit in one CTA.
size_t solve_fill_args(const pa_ctx* ctx, int C, int gen0, int G, const uint8_t* pop_in,
                       uint8_t* pop_out, void* fit_out, uint8_t* best_row, double* best_fit,
                       void* args_out, bool latency, int threads) {
  const pa_config& c = ctx->cfg;
  if (C > c.N || ctx->t32.streamed) return 0;
  const SolveShape s = solve_shape(ctx, C, latency ? kSoloMaxNP : kBatchMaxNP,
                                   threads == kSmallCtaThreads ? kSmallCtaThreads : kSolveThreads);
  if (s.smem > (size_t)kSmemBudget - 64 * 4 - 16) return 0;
  SolveArgs a{};
  a.pop_in = pop_in;
  a.pop_out = pop_out;
  a.fit_out = fit_out;
  a.best_row = best_row;
  a.best_fit = best_fit;
  a.N = c.N;
  a.L = c.L;
  a.K = c.K;
  a.E = c.E;
  a.tour = c.tour;
  a.pc_thresh = c.pc_thresh;
  a.pm_thresh = c.pm_thresh;
  a.seed = c.seed;
  a.gen0 = gen0;
  a.G = G;
  a.NT = s.NT;
  a.MS = s.MS;
  a.XO = s.XO;
  a.NTT = s.NTT;
  a.nblk = s.nblk;
  a.CH = s.CH;
  a.tab = ctx->t32.tab;
  a.own = ctx->t32.own;
  a.bn = ctx->t32.bn;
  a.RS = ctx->t32.RS;
  a.tab_floats = (((int64_t)c.L * c.K * ctx->t32.RS + 3) / 4) * 4;
  a.M32 = ctx->t32.M;
  a.pc32 = ctx->t32.pc;
  a.beta = ctx->beta64;
  a.bnc = ctx->bnc64;
  a.M64 = c.M;
  a.pc64 = ctx->pc;
  a.fin = c.mode == PA_SINR_FINITE_M;
  a.obj = c.objective;
  std::memcpy(args_out, &a, sizeof a);
  return s.smem;
}

// Set the completion-time stamp of an argument record (a SolveArgs).
void solve_args_set_stamp(void* args, unsigned long long* stamp) {
  static_cast<SolveArgs*>(args)->stamp = stamp;
}

// Clusters of size C that can be resident at once for the batched kernel of
// proto's variant with this shared memory (0 when none).
// Cached per (device, kernel variant, cluster size, shared memory): the
// occupancy query costs host time on every scheduling tick otherwise.
int solve_batch_max_clusters(const pa_ctx* proto, int C, size_t smem, bool latency, int threads) {
  struct Key {
    int dev, prec, fin, nj, vec, C, lat, thr;
    size_t smem;
    bool operator<(const Key& o) const {
      return std::tie(dev, prec, fin, nj, vec, C, lat, thr, smem) <
             std::tie(o.dev, o.prec, o.fin, o.nj, o.vec, o.C, o.lat, o.thr, o.smem);
    }
  };
  static std::map<Key, int> cache;
  static std::mutex mu;
  const Key k{proto->device, proto->cfg.prec, proto->cfg.mode, proto->t32.NJ, proto->t32.vec, C,
              latency ? 1 : 0, threads, smem};
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(k);
    if (it != cache.end()) return it->second;
  }
  int m = 0;
  if (dispatch_any(latency, threads, proto, C, 1, nullptr, 0, nullptr, smem, true, &m, nullptr) !=
      cudaSuccess)
    return 0;
  std::lock_guard<std::mutex> lock(mu);
  cache[k] = m;
  return m;
}

// Persistent batched solve of n instances sharing proto's kernel variant:
// d_args holds their SolveArgs (cluster size C), d_counter must be zero.
cudaError_t launch_solve_batch(const pa_ctx* proto, int C, int clusters, const void* d_args, int n,
                               int* d_counter, size_t smem, cudaStream_t st, bool latency,
                               int threads) {
  return dispatch_any(latency, threads, proto, C, clusters, static_cast<const SolveArgs*>(d_args),
                      n, d_counter, smem, false, nullptr, st);
}

}  // namespace pa
