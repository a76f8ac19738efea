// pa_solve_batch_small.cu -- the batched solve kernel with 256-thread CTAs:
// four CTAs, and so four instances (or four clusters' shares of them), are
// resident per SM, which overlaps one instance's GA phase and barriers with
// another's evaluation.  The batch autotuner times this shape against
// 1024-thread CTAs for every kernel-variant group.  A translation unit of
// its own so that it compiles in parallel with the other variants.
#include "pa_solve_batch.cuh"

namespace pa {

cudaError_t dispatch_batch_small(const pa_ctx* proto, int C, int clusters, const void* d, int n,
                                 int* ctr, size_t smem, bool q, int* mc, cudaStream_t st) {
  return dispatch_batch<kBatchMaxNP, kSmallCtaThreads>(proto, C, clusters,
                                                      static_cast<const SolveArgs*>(d), n, ctr,
                                                      smem, q, mc, st);
}

}  // namespace pa
