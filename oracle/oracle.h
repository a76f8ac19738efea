/*
 * oracle.h -- plain, slow FP64 CPU oracle for the K-means-seeded 2D genetic
 * algorithm for massive-MIMO pilot assignment (arXiv 2511.20511).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Notation (paper Sec. 3): L cells, K users per cell, K pilots per cell.
 *   beta[(j*L + l)*K + k]  large-scale fading of user k of cell l at BS j
 *                          (Eq. 2; index order of the channel h_ijk, Eq. 1)
 *   X[l*K + k]             pilot of user k of cell l; each row l is a
 *                          permutation of 0..K-1 (Sec. 4.1 chromosome)
 *
 * Every function is pinned by the tests under tests/ (test_oracle_*.py):
 * hand-computed values, closed forms, invariants, brute force, scikit-learn's
 * Lloyd iteration, numpy's Philox, chi-square tests of the random draws.
 * Parity unpinned: whether the GA as a whole reproduces the paper's
 * convergence figures (Fig. 4, 82 s / 116 s) -- the paper's runs, seeds and
 * data are not available; every function here is pinned.
 */
#ifndef PA_ORACLE_H
#define PA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SINR model selector. */
enum { OR_ASYMPTOTIC = 0, OR_FINITE_M = 1 };

/* Objective: the sum SE of Eq. 7, or the smallest per-user SINR (the
   max-min SIR objective stated in Sec. 2). */
enum { OR_OBJ_SUM_SE = 0, OR_OBJ_MIN_SINR = 1 };

/* Parameters of the SINR model.  Only read in OR_FINITE_M mode except mode
   and objective. */
typedef struct {
  int32_t mode;   /* OR_ASYMPTOTIC (Eq. 4-5) or OR_FINITE_M (Eq. 3 reading) */
  int32_t tau_p;  /* pilot length */
  double M;       /* BS antennas */
  double rho;     /* transmit SNR scale (power / noise unit) */
  double sigma2;  /* noise variance */
  int32_t objective; /* OR_OBJ_SUM_SE or OR_OBJ_MIN_SINR */
  int32_t pad0;
} or_sinr_params;

/* GA parameters (Alg. 1): elitism, tournament with replacement, row-wise
   one-cut crossover, per-row swap mutation. */
typedef struct {
  int32_t N;          /* population size */
  int32_t E;          /* elites */
  int32_t tour;       /* tournament size */
  int32_t pad0;
  uint64_t pc_thresh; /* crossover  iff draw <  pc_thresh  (0..2^32) */
  uint64_t pm_thresh; /* row swap   iff draw <  pm_thresh  (0..2^32) */
  uint64_t seed;
} or_ga_params;

/* Philox4x64-10 block function (Salmon et al., SC'11). */
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* 32-bit draw number d of the stream (seed; slot, gen, tag). */
uint32_t or_draw32(uint64_t seed, uint64_t slot, uint64_t gen, uint64_t tag, uint32_t d);

/* log2 by the atanh series (Abramowitz & Stegun 4.1.27), x >= 1. */
double or_log2_det(double x);

/* Fitness of one chromosome: sum-SE, Eq. 6 with per-user SE of Eq. 5
 * (OR_OBJ_SUM_SE), or the smallest per-user SINR (OR_OBJ_MIN_SINR, Sec. 2).
 * sinr_out / se_out (optional, L*K) receive the per-user values. */
double or_fitness(const double* beta, int32_t L, int32_t K, const uint8_t* X,
                  const or_sinr_params* sp, double* sinr_out, double* se_out);

/* Fitness of n chromosomes stored back to back (n*L*K bytes). */
void or_fitness_batch(const double* beta, int32_t L, int32_t K, const uint8_t* pop,
                      int64_t n, const or_sinr_params* sp, double* fit);

/* One GA generation (Alg. 1 selection/crossover/mutation with elitism). */
void or_ga_step(const uint8_t* pop, const double* fit, int32_t L, int32_t K,
                const or_ga_params* gp, int32_t gen, uint8_t* next);

/* K-means features: user position relative to its own BS, integer mm. */
void or_features(int32_t L, int32_t K, const int32_t* user_xy_mm,
                 const int32_t* bs_xy_mm, int64_t* fx, int64_t* fy);

/* Lloyd's K-means with k clusters over U points; returns assignment passes. */
int32_t or_kmeans(int32_t U, const int64_t* fx, const int64_t* fy, int32_t k,
                  int32_t max_iter, uint64_t seed, int32_t* label, double* cx, double* cy);

/* Squared distance of a point to a centroid, in the order K-means uses. */
double or_dist2(int64_t fx, int64_t fy, double cx, double cy);

/* Population seeding from K-means labels (label == NULL: all random). */
void or_seed_population(int32_t L, int32_t K, const int32_t* label, const int64_t* fx,
                        const int64_t* fy, const double* cx, const double* cy,
                        int32_t N, int32_t n_seeded, uint64_t seed, uint8_t* pop);

/* Whole solve: seed, G generations, final evaluation.  hist_best (G+1)
 * receives the best fitness of each evaluated generation. */
void or_solve(const double* beta, int32_t L, int32_t K, const or_sinr_params* sp,
              const or_ga_params* gp, const int32_t* user_xy_mm, const int32_t* bs_xy_mm,
              int32_t kmeans_k, int32_t kmeans_max_iter, int32_t n_seeded, int32_t G,
              uint8_t* pop_out, double* fit_out, uint8_t* best_out, double* best_fit,
              double* hist_best);

/* ---- PK-means GA (Alg. 2): islands of the population found by K-means.
 * A chromosome is represented by its one-hot pilot indicators (one K-vector
 * per user), so the squared distance between two chromosomes is twice the
 * number of users whose pilots differ, and a centroid holds, per user, the
 * fraction of the cluster's members giving that user each pilot.  Integer
 * arithmetic throughout (requires N <= 4096, L*K <= 4096). */

/* Lloyd's K-means of the N chromosomes into C clusters (Alg. 2 "Apply
 * K-means"); initial centroids are C distinct members drawn by a partial
 * Fisher-Yates shuffle keyed by generation gen (init_out, optional, C:
 * their indices).  label (N) out; returns the number of assignment passes. */
int32_t or_pop_kmeans(const uint8_t* pop, int32_t N, int32_t L, int32_t K, int32_t C,
                      int32_t max_iter, uint64_t seed, int32_t gen, int32_t* label,
                      int32_t* init_out);

/* One generation of the island GA (Alg. 2 loop body): each cluster c of
 * label evolves on its own slots -- elites, tournaments over its members,
 * crossover, mutation -- with the draws of or_ga_step. */
void or_island_step(const uint8_t* pop, const double* fit, int32_t L, int32_t K,
                    const or_ga_params* gp, int32_t gen, const int32_t* label, int32_t C,
                    uint8_t* next);

/* Whole island solve: seeding as or_solve, then G generations, the
 * population re-clustered into C islands every R generations (Sec. 6.1:
 * every three) with at most iters passes.  label_out (N, optional): the
 * last clustering. */
void or_solve_islands(const double* beta, int32_t L, int32_t K, const or_sinr_params* sp,
                      const or_ga_params* gp, const int32_t* user_xy_mm, const int32_t* bs_xy_mm,
                      int32_t kmeans_k, int32_t kmeans_max_iter, int32_t n_seeded, int32_t G,
                      int32_t C, int32_t R, int32_t iters, uint8_t* pop_out, double* fit_out,
                      uint8_t* best_out, double* best_fit, double* hist_best,
                      int32_t* label_out);

/* Exhaustive search (EX-PA): row 0 fixed to the identity unless all_rows. */
double or_exhaustive(const double* beta, int32_t L, int32_t K, const or_sinr_params* sp,
                     int32_t all_rows, uint8_t* best_X, int64_t* n_evaluated);

#ifdef __cplusplus
}
#endif
#endif
