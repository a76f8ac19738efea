// pa_solve_batch_lat.cu -- the batched solve kernel with the one-instance
// kernel's column split (more threads per pilot, shorter evaluation passes):
// for a few concurrent instances, where each generation's latency matters
// more than instruction throughput.  A translation unit of its own so that
// it compiles in parallel with the throughput variant.
#include "pa_solve_batch.cuh"

namespace pa {

cudaError_t dispatch_batch_latency(const pa_ctx* proto, int C, int clusters, const void* d, int n,
                                   int* ctr, size_t smem, bool q, int* mc, cudaStream_t st) {
  return dispatch_batch<kSoloMaxNP, kSolveThreads>(proto, C, clusters, static_cast<const SolveArgs*>(d), n, ctr,
                                    smem, q, mc, st);
}

}  // namespace pa
