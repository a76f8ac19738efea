// pa_solve.cu -- whole GA runs (Alg. 1 loop) in one launch of one
// thread-block cluster per instance.
//
// Each of the C CTAs of the cluster owns NT consecutive members of the
// population in its shared memory, next to its own copy of the instance
// tables.  One generation:
//   1. every CTA evaluates its members (Eq. 3-6) and writes their fitness
//      into every CTA's copy of the fitness vector (distributed shared
//      memory stores);
//   2. one cluster barrier (release/acquire): all fitness values and all
//      members of this generation are visible cluster-wide;
//   3. every CTA builds its own child slots (one warp per child): elites by
//      (fitness desc, index asc), tournaments over the local fitness copy,
//      parent rows read from their owners' shared memory, row-wise one-cut
//      crossover, per-row swap mutation -- the same draws as k_ga_step.
// Populations and fitness vectors are double-buffered, so one barrier per
// generation suffices: a buffer is rewritten one generation after it was
// read, and every CTA finished that read before arriving at the barrier the
// writer has passed.  The barrier is the hardware cluster barrier (no
// software spin).  After G generations the final population is evaluated,
// written to global memory with its fitness, and CTA 0 selects the best
// member.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>

#include "pa_solve_launch.cuh"

namespace pa {

// Run G generations from pop_in into pop_out (fitness of the final
// population to fit_out; best member to best_row/best_fit when given) in
// one cluster launch.  The cluster size is the largest of 16 (non-portable),
// 8, 4, 2, 1 CTAs that can be resident with this shared memory, never more
// CTAs than members; it is found on the first call and kept in the context.
// Returns cudaErrorNotSupported when no shape fits (the caller then runs
// the per-generation kernels).  With isl given: island mode (Alg. 2), the
// islands of isl_label with member lists isl (E <= 8 only).
cudaError_t launch_solve(pa_ctx* ctx, const uint8_t* pop_in, uint8_t* pop_out, int gen0, int G,
                         void* fit_out, uint8_t* best_row, double* best_fit, cudaStream_t st,
                         int32_t* isl_label, IslandLists* isl, bool isl_km) {
  if (ctx->solve_C == 0 || ctx->t32.streamed) return cudaErrorNotSupported;
  const pa_config& c = ctx->cfg;
  if ((c.islands >= 2) != (isl != nullptr)) return cudaErrorNotSupported;
  if (isl && c.E > kSmallE) return cudaErrorNotSupported;
  static const int sizes[] = {16, 8, 4, 2, 1};
  for (int C : sizes) {
    if (ctx->solve_C > 0 && C != ctx->solve_C) continue;
    if (C > c.N) continue;
    SolveShape s = solve_shape(ctx, C, kSoloMaxNP, kSolveThreads);
    if (s.smem > (size_t)kSmemBudget - 64 * 4) continue;
    SolveArgs a{};
    if (isl_km) {  // K-means arrays after the solve's (KmView of pa_island_kmeans.cuh)
      const size_t N4 = (size_t)((c.N + 3) & ~3), LK = (size_t)c.L * c.K;
      const int W = (int)((LK + 3) / 4), NP = c.N | 1, CWp = ((c.islands + 1) / 2) | 1;
      const int Nr = (c.N + C - 1) / C, groups = (Nr + 31) / 32;
      auto r16 = [](size_t v) { return (v + 15) & ~size_t(15); };
      bool fits = false;
      for (int us = std::max(1, std::min({kKmSplits, kSolveThreads / 32 / groups, W})); us >= 1;
           --us) {
        size_t b = r16(s.smem);
        a.o_ksh = (int)b;
        b = r16(b + sizeof(KmShared));
        a.o_kpw = (int)b;
        b = r16(b + 4 * (size_t)W * NP);
        a.o_kcnt = (int)b;
        b = r16(b + 4 * LK * c.K * CWp);
        a.o_klab = (int)b;
        b += 4 * 2 * N4;  // labels, initial permutation
        a.o_kchg = (int)b;
        b += 4 * 2 * N4;
        a.o_kgchg = (int)b;
        b += 4 * N4;
        a.o_ksb = (int)b;
        if (us > 1) b += 4 * (size_t)us * c.islands * Nr;
        a.isl_us = us;
        if (r16(b) <= (size_t)kSmemBudget - 64 * 4) {
          s.smem = r16(b);
          fits = true;
          break;
        }
      }
      if (!fits) continue;  // no room beside the solve at this cluster size
    }
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
    if (isl) {
      a.isl_label = isl_label;
      a.isl_off = isl->off;
      a.isl_list = isl->list;
      a.isl_pos = isl->pos;
      a.isl_C = c.islands;
      if (isl_km) {
        a.isl_km = 1;
        a.isl_R = c.recluster;
        a.isl_iter = c.island_iter;
        a.isl_fresh = ctx->isl_valid ? 0 : 1;
        a.isl_label_out = isl_label;
        a.isl_off_out = isl->off;
        a.isl_list_out = isl->list;
        a.isl_pos_out = isl->pos;
      }
    }
    const bool fin = a.fin;
    const bool chk = ctx->solve_C < 0;
    cudaError_t e;
    if (isl)
      e = solve_island_dispatch(&a, &s, chk, c.prec == PA_FP64, ctx->t32.vec, fin, ctx->t32.NJ,
                                st);
    else if (c.prec == PA_FP64)
      e = run_solve<double, 4, 2, false, false>(a, s, chk, st);
    else if (ctx->t32.vec == 2)
      e = fin ? pick_solve<float, 2, true, false>(ctx->t32.NJ, a, s, chk, st)
              : pick_solve<float, 2, false, false>(ctx->t32.NJ, a, s, chk, st);
    else
      e = fin ? pick_solve<float, 1, true, false>(ctx->t32.NJ, a, s, chk, st)
              : pick_solve<float, 1, false, false>(ctx->t32.NJ, a, s, chk, st);
    if (e == cudaErrorNotSupported) continue;
    if (e == cudaSuccess) ctx->solve_C = C;
    return e;
  }
  if (!isl_km) ctx->solve_C = 0;  // (the caller of isl_km falls back to launches per block)
  return cudaErrorNotSupported;
}

// ------------------------------------------------------------------ batches

}  // namespace pa
