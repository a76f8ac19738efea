// pa_solve_island.cu -- the fused solve in island mode (Alg. 2): tournaments
// and elites within each member's island, and (isl_km) the population
// K-means every few generations inside the same cluster launch, so that a
// whole island solve is one launch (k_solve with ISL; the launch and the
// kernel are those of pa_solve_launch.cuh, instantiated here).
#include "pa_solve_launch.cuh"

namespace pa {

cudaError_t solve_island_dispatch(const void* args, const void* shape, bool check_fit, bool f64,
                                  int vec, bool fin, int NJ, cudaStream_t st) {
  const SolveArgs& a = *static_cast<const SolveArgs*>(args);
  const SolveShape& s = *static_cast<const SolveShape*>(shape);
  if (f64) return run_solve<double, 4, 2, false, true>(a, s, check_fit, st);
  if (vec != 2) return cudaErrorNotSupported;
  return fin ? pick_solve<float, 2, true, true>(NJ, a, s, check_fit, st)
             : pick_solve<float, 2, false, true>(NJ, a, s, check_fit, st);
}

}  // namespace pa
