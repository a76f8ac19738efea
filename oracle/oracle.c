/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Written to be checked against the paper by eye: straight loops, one IEEE
 * operation per step, fixed summation order, no blocking or fusion.  Compile
 * with -ffp-contract=off so that no multiply-add is fused.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the 4x64 S-box with key bumps.  */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1  */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(PHILOX_M0, c0, &hi0, &lo0);
    mulhilo64(PHILOX_M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw d of a stream: block d/8 of the counter (d>>3, slot, gen, tag) under
 * key (seed, 0); 64-bit word (d>>1)&3 of that block; low half for even d,
 * high half for odd d. */
uint32_t or_draw32(uint64_t seed, uint64_t slot, uint64_t gen, uint64_t tag, uint32_t d) {
  uint64_t ctr[4] = {(uint64_t)(d >> 3), slot, gen, tag};
  uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  or_philox4x64_10(ctr, key, out);
  uint64_t w = out[(d >> 1) & 3u];
  return (d & 1u) ? (uint32_t)(w >> 32) : (uint32_t)(w & 0xFFFFFFFFu);
}

/* Uniform integer in [0, n) from a 32-bit draw (multiply-shift). */
static uint32_t below(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* Stream tags. */
enum { TAG_SEED = 1, TAG_KMEANS = 2, TAG_GA = 3, TAG_ISLAND = 4 };

/* ------------------------------------------------------------------------ */
/* log2 by the series ln m = 2 * sum_{n>=0} s^(2n+1) / (2n+1), s=(m-1)/(m+1) */
/* (Abramowitz & Stegun 4.1.27), after splitting x = m * 2^e with m in      */
/* [sqrt(1/2), sqrt(2)).  Terms up to s^23, Horner from the highest.         */
/* ------------------------------------------------------------------------ */
double or_log2_det(double x) {
  if (isinf(x)) return x;
  int E;
  double f = frexp(x, &E); /* x = f * 2^E, f in [0.5, 1) */
  double m;
  int e;
  if (f < 0.70710678118654752440) {
    m = f * 2.0;
    e = E - 1;
  } else {
    m = f;
    e = E;
  }
  double s = (m - 1.0) / (m + 1.0);
  double t = s * s;
  double p = 1.0 / 23.0;
  p = p * t + 1.0 / 21.0;
  p = p * t + 1.0 / 19.0;
  p = p * t + 1.0 / 17.0;
  p = p * t + 1.0 / 15.0;
  p = p * t + 1.0 / 13.0;
  p = p * t + 1.0 / 11.0;
  p = p * t + 1.0 / 9.0;
  p = p * t + 1.0 / 7.0;
  p = p * t + 1.0 / 5.0;
  p = p * t + 1.0 / 3.0;
  p = p * t + 1.0;
  double ln_m = (2.0 * s) * p;
  return (double)e + ln_m * 1.44269504088896340736; /* 1 / ln 2 */
}

/* ------------------------------------------------------------------------ */
/* Fitness (Sec. 3, Eq. 3-7).                                                */
/* ------------------------------------------------------------------------ */

/* inv[l*K + p] = user of cell l that holds pilot p. */
static void inverse_rows(const uint8_t* X, int32_t L, int32_t K, int32_t* inv) {
  for (int32_t l = 0; l < L; ++l)
    for (int32_t k = 0; k < K; ++k) inv[l * K + X[l * K + k]] = k;
}

static double beta_at(const double* beta, int32_t L, int32_t K, int32_t j, int32_t l,
                      int32_t k) {
  return beta[((int64_t)j * L + l) * K + k];
}

/*
 * For user k of cell j holding pilot p = X[j][k], the users sharing pilot p
 * in the other cells l != j are inv[l][p] (pilots are reused across cells,
 * Sec. 3.1; search space K!^(L-1), Sec. 3.3).  Their gains at BS j give the
 * coherent pilot-contamination interference of Eq. 4-5:
 *     S2 = sum_{l != j, ascending} beta[j][l][inv[l][p]]^2
 *   ASYMPTOTIC (Eq. 4-5):  sinr = beta[j][j][k]^2 / S2
 *   FINITE_M  (reading of Eq. 3 with MMSE pilot estimates, MR combining):
 *     S1   = sum_{l ascending}  beta[j][l][inv[l][p]]           (incl. own)
 *     B_j  = sum_l sum_k beta[j][l][k]                           (all users)
 *     sinr = M beta_jjk^2 / (M S2 + (B_j + sigma2/rho) (S1 + sigma2/(tau_p rho)))
 *   SE = log2(1 + sinr)  (Eq. 5),   fitness = sum_j (sum_k SE)   (Eq. 6).
 * The max-min objective of Sec. 2 instead takes fitness = the smallest sinr
 * over all users (j ascending, k ascending; a minimum has no rounding).
 */
double or_fitness(const double* beta, int32_t L, int32_t K, const uint8_t* X,
                  const or_sinr_params* sp, double* sinr_out, double* se_out) {
  int32_t* inv = (int32_t*)malloc(sizeof(int32_t) * (size_t)L * (size_t)K);
  inverse_rows(X, L, K, inv);
  const int finite = (sp->mode == OR_FINITE_M);
  const double nc = sp->sigma2 / sp->rho;
  const double pc = sp->sigma2 / ((double)sp->tau_p * sp->rho);
  double fitness = 0.0;
  double min_sinr = INFINITY;
  for (int32_t j = 0; j < L; ++j) {
    double b_j = 0.0;
    if (finite) {
      for (int32_t l = 0; l < L; ++l)
        for (int32_t k = 0; k < K; ++k) b_j = b_j + beta_at(beta, L, K, j, l, k);
    }
    double cell_sum = 0.0;
    for (int32_t k = 0; k < K; ++k) {
      int32_t p = X[j * K + k];
      double s2 = 0.0;
      double s1 = 0.0;
      for (int32_t l = 0; l < L; ++l) {
        double b = beta_at(beta, L, K, j, l, inv[l * K + p]);
        if (finite) s1 = s1 + b;
        if (l != j) s2 = s2 + b * b;
      }
      double own = beta_at(beta, L, K, j, j, k);
      double own2 = own * own;
      double sinr;
      if (finite) {
        double num = sp->M * own2;
        double den = sp->M * s2 + (b_j + nc) * (s1 + pc);
        sinr = num / den;
      } else {
        sinr = own2 / s2;
      }
      double se = or_log2_det(1.0 + sinr);
      if (sinr_out) sinr_out[j * K + k] = sinr;
      if (se_out) se_out[j * K + k] = se;
      cell_sum = cell_sum + se;
      if (sinr < min_sinr) min_sinr = sinr;
    }
    fitness = fitness + cell_sum;
  }
  free(inv);
  return sp->objective == OR_OBJ_MIN_SINR ? min_sinr : fitness;
}

void or_fitness_batch(const double* beta, int32_t L, int32_t K, const uint8_t* pop,
                      int64_t n, const or_sinr_params* sp, double* fit) {
  for (int64_t i = 0; i < n; ++i)
    fit[i] = or_fitness(beta, L, K, pop + i * (int64_t)L * K, sp, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* GA generation (Alg. 1: selection, crossover, mutation; elitism, Sec. 1). */
/* ------------------------------------------------------------------------ */

/* a is better than b: higher fitness, ties to the lower index. */
static int better(const double* fit, int32_t a, int32_t b) {
  if (fit[a] > fit[b]) return 1;
  if (fit[a] < fit[b]) return 0;
  return a < b;
}

/* Tournament of size tour drawn with replacement from draws first..first+tour-1. */
static int32_t tournament(const double* fit, int32_t N, int32_t tour, uint64_t seed,
                          int32_t slot, int32_t gen, uint32_t first) {
  int32_t best = (int32_t)below(or_draw32(seed, slot, gen, TAG_GA, first), (uint32_t)N);
  for (int32_t t = 1; t < tour; ++t) {
    int32_t c = (int32_t)below(or_draw32(seed, slot, gen, TAG_GA, first + t), (uint32_t)N);
    if (better(fit, c, best)) best = c;
  }
  return best;
}

/* Swap two distinct positions of one row chosen by draws ui, uj. */
static void swap_two(uint8_t* row, int32_t K, uint32_t ui, uint32_t uj) {
  if (K < 2) return;
  int32_t i = (int32_t)below(ui, (uint32_t)K);
  int32_t jj = (int32_t)below(uj, (uint32_t)(K - 1));
  int32_t j = jj + (jj >= i ? 1 : 0);
  uint8_t tmp = row[i];
  row[i] = row[j];
  row[j] = tmp;
}

void or_ga_step(const uint8_t* pop, const double* fit, int32_t L, int32_t K,
                const or_ga_params* gp, int32_t gen, uint8_t* next) {
  const int32_t N = gp->N, E = gp->E, T = gp->tour;
  const int64_t LK = (int64_t)L * K;
  /* Elites: the E best by (fitness desc, index asc), copied unchanged. */
  char* taken = (char*)calloc((size_t)N, 1);
  for (int32_t e = 0; e < E; ++e) {
    int32_t best = -1;
    for (int32_t i = 0; i < N; ++i)
      if (!taken[i] && (best < 0 || better(fit, i, best))) best = i;
    taken[best] = 1;
    memcpy(next + e * LK, pop + best * LK, (size_t)LK);
  }
  free(taken);
  /* Children: two tournaments, row-wise one-cut crossover, row swap mutation. */
  for (int32_t n = E; n < N; ++n) {
    uint8_t* child = next + n * LK;
    int32_t a = tournament(fit, N, T, gp->seed, n, gen, 0);
    int32_t b = tournament(fit, N, T, gp->seed, n, gen, (uint32_t)T);
    uint32_t u_cross = or_draw32(gp->seed, n, gen, TAG_GA, (uint32_t)(2 * T));
    uint32_t u_cut = or_draw32(gp->seed, n, gen, TAG_GA, (uint32_t)(2 * T + 1));
    int32_t cut = L; /* rows < cut from a, rows >= cut from b */
    if ((uint64_t)u_cross < gp->pc_thresh) cut = 1 + (int32_t)below(u_cut, (uint32_t)(L - 1));
    for (int32_t l = 0; l < L; ++l) {
      const uint8_t* src = (l < cut) ? pop + a * LK : pop + b * LK;
      memcpy(child + l * K, src + l * K, (size_t)K);
    }
    for (int32_t l = 0; l < L; ++l) {
      uint32_t base = (uint32_t)(2 * T + 2 + 3 * l);
      uint32_t u_mut = or_draw32(gp->seed, n, gen, TAG_GA, base);
      uint32_t ui = or_draw32(gp->seed, n, gen, TAG_GA, base + 1);
      uint32_t uj = or_draw32(gp->seed, n, gen, TAG_GA, base + 2);
      if ((uint64_t)u_mut < gp->pm_thresh) swap_two(child + l * K, K, ui, uj);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* K-means (Sec. 4.1, Alg. 1 "Apply K-means clustering"; Table 3 O(NCKd)).  */
/* ------------------------------------------------------------------------ */
void or_features(int32_t L, int32_t K, const int32_t* user_xy_mm, const int32_t* bs_xy_mm,
                 int64_t* fx, int64_t* fy) {
  for (int32_t l = 0; l < L; ++l)
    for (int32_t k = 0; k < K; ++k) {
      int32_t u = l * K + k;
      fx[u] = (int64_t)user_xy_mm[2 * u] - (int64_t)bs_xy_mm[2 * l];
      fy[u] = (int64_t)user_xy_mm[2 * u + 1] - (int64_t)bs_xy_mm[2 * l + 1];
    }
}

double or_dist2(int64_t fx, int64_t fy, double cx, double cy) {
  double dx = (double)fx - cx;
  double dy = (double)fy - cy;
  return dx * dx + dy * dy;
}

int32_t or_kmeans(int32_t U, const int64_t* fx, const int64_t* fy, int32_t k,
                  int32_t max_iter, uint64_t seed, int32_t* label, double* cx, double* cy) {
  /* Initial centroids: k distinct points by a partial Fisher-Yates shuffle. */
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)U);
  for (int32_t i = 0; i < U; ++i) idx[i] = i;
  for (int32_t i = 0; i < k; ++i) {
    int32_t j = i + (int32_t)below(or_draw32(seed, 0, 0, TAG_KMEANS, (uint32_t)i),
                                   (uint32_t)(U - i));
    int32_t t = idx[i];
    idx[i] = idx[j];
    idx[j] = t;
    cx[i] = (double)fx[idx[i]];
    cy[i] = (double)fy[idx[i]];
  }
  free(idx);
  for (int32_t u = 0; u < U; ++u) label[u] = -1;
  int64_t* sx = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
  int64_t* sy = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
  int32_t passes = 0;
  for (int32_t it = 0; it < max_iter; ++it) {
    /* Assignment: nearest centroid, ties to the lower centroid index. */
    int64_t changed = 0;
    for (int32_t u = 0; u < U; ++u) {
      int32_t best = 0;
      double bd = or_dist2(fx[u], fy[u], cx[0], cy[0]);
      for (int32_t c = 1; c < k; ++c) {
        double d = or_dist2(fx[u], fy[u], cx[c], cy[c]);
        if (d < bd) {
          bd = d;
          best = c;
        }
      }
      if (label[u] != best) changed++;
      label[u] = best;
    }
    passes++;
    if (changed == 0 || it == max_iter - 1) break;
    /* Update: exact integer sums per cluster, one division; empty keeps. */
    for (int32_t c = 0; c < k; ++c) sx[c] = sy[c] = cnt[c] = 0;
    for (int32_t u = 0; u < U; ++u) {
      sx[label[u]] += fx[u];
      sy[label[u]] += fy[u];
      cnt[label[u]] += 1;
    }
    for (int32_t c = 0; c < k; ++c)
      if (cnt[c] > 0) {
        cx[c] = (double)sx[c] / (double)cnt[c];
        cy[c] = (double)sy[c] / (double)cnt[c];
      }
  }
  free(sx);
  free(sy);
  free(cnt);
  return passes;
}

/* ------------------------------------------------------------------------ */
/* Population seeding from the clustering (Sec. 1 contribution 2; Alg. 1).  */
/* ------------------------------------------------------------------------ */

/* A*: in each cell, users in order of (distance to own centroid, index) take
 * pilot = label when that pilot is still free; the others take the free
 * pilots in ascending order. */
static void kmeans_assignment(int32_t L, int32_t K, const int32_t* label, const int64_t* fx,
                              const int64_t* fy, const double* cx, const double* cy,
                              uint8_t* out) {
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  double* dist = (double*)malloc(sizeof(double) * (size_t)K);
  int32_t* deferred = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  char* used = (char*)malloc((size_t)K);
  for (int32_t l = 0; l < L; ++l) {
    for (int32_t k = 0; k < K; ++k) {
      int32_t u = l * K + k;
      dist[k] = or_dist2(fx[u], fy[u], cx[label[u]], cy[label[u]]);
      order[k] = k;
    }
    /* insertion sort by (dist, k) */
    for (int32_t i = 1; i < K; ++i) {
      int32_t v = order[i];
      int32_t j = i - 1;
      while (j >= 0 && (dist[order[j]] > dist[v] || (dist[order[j]] == dist[v] && order[j] > v))) {
        order[j + 1] = order[j];
        j--;
      }
      order[j + 1] = v;
    }
    memset(used, 0, (size_t)K);
    int32_t nd = 0;
    for (int32_t i = 0; i < K; ++i) {
      int32_t k = order[i];
      int32_t p = label[l * K + k];
      if (!used[p]) {
        used[p] = 1;
        out[l * K + k] = (uint8_t)p;
      } else {
        deferred[nd++] = k;
      }
    }
    int32_t next_free = 0;
    for (int32_t i = 0; i < nd; ++i) {
      while (used[next_free]) next_free++;
      used[next_free] = 1;
      out[l * K + deferred[i]] = (uint8_t)next_free;
    }
  }
  free(order);
  free(dist);
  free(deferred);
  free(used);
}

/* Uniformly random row: identity, then Fisher-Yates from the top. */
static void random_row(uint8_t* row, int32_t K, uint64_t seed, int32_t n, uint32_t first) {
  for (int32_t k = 0; k < K; ++k) row[k] = (uint8_t)k;
  for (int32_t t = 0; t < K - 1; ++t) {
    int32_t i = K - 1 - t;
    int32_t j = (int32_t)below(or_draw32(seed, n, 0, TAG_SEED, first + t), (uint32_t)(i + 1));
    uint8_t tmp = row[i];
    row[i] = row[j];
    row[j] = tmp;
  }
}

void or_seed_population(int32_t L, int32_t K, const int32_t* label, const int64_t* fx,
                        const int64_t* fy, const double* cx, const double* cy, int32_t N,
                        int32_t n_seeded, uint64_t seed, uint8_t* pop) {
  const int64_t LK = (int64_t)L * K;
  if (label == NULL) n_seeded = 0;
  uint8_t* astar = (uint8_t*)malloc((size_t)LK);
  if (n_seeded > 0) kmeans_assignment(L, K, label, fx, fy, cx, cy, astar);
  for (int32_t n = 0; n < N; ++n) {
    uint8_t* X = pop + n * LK;
    if (n < n_seeded) {
      memcpy(X, astar, (size_t)LK);
      if (n > 0) {
        for (int32_t l = 0; l < L; ++l) {
          uint32_t u_do = or_draw32(seed, n, 0, TAG_SEED, (uint32_t)(3 * l));
          uint32_t ui = or_draw32(seed, n, 0, TAG_SEED, (uint32_t)(3 * l + 1));
          uint32_t uj = or_draw32(seed, n, 0, TAG_SEED, (uint32_t)(3 * l + 2));
          if (u_do < 0x80000000u) swap_two(X + l * K, K, ui, uj);
        }
      }
    } else {
      for (int32_t l = 0; l < L; ++l)
        random_row(X + l * K, K, seed, n, (uint32_t)(l * (K - 1 > 0 ? K - 1 : 0)));
    }
  }
  free(astar);
}

/* ------------------------------------------------------------------------ */
/* Whole solve (Alg. 1 loop with K-means seeding).                           */
/* ------------------------------------------------------------------------ */
static int32_t argbest(const double* fit, int32_t N) {
  int32_t best = 0;
  for (int32_t i = 1; i < N; ++i)
    if (better(fit, i, best)) best = i;
  return best;
}

/* Initial population of a solve: K-means seeding with positions, else all
 * random rows. */
static void initial_population(int32_t L, int32_t K, const or_ga_params* gp,
                               const int32_t* user_xy_mm, const int32_t* bs_xy_mm,
                               int32_t kmeans_k, int32_t kmeans_max_iter, int32_t n_seeded,
                               uint8_t* pop) {
  const int32_t N = gp->N;
  const int32_t U = L * K;
  if (user_xy_mm != NULL && bs_xy_mm != NULL) {
    int64_t* fx = (int64_t*)malloc(sizeof(int64_t) * (size_t)U);
    int64_t* fy = (int64_t*)malloc(sizeof(int64_t) * (size_t)U);
    int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)U);
    double* cx = (double*)malloc(sizeof(double) * (size_t)kmeans_k);
    double* cy = (double*)malloc(sizeof(double) * (size_t)kmeans_k);
    or_features(L, K, user_xy_mm, bs_xy_mm, fx, fy);
    or_kmeans(U, fx, fy, kmeans_k, kmeans_max_iter, gp->seed, label, cx, cy);
    or_seed_population(L, K, label, fx, fy, cx, cy, N, n_seeded, gp->seed, pop);
    free(fx);
    free(fy);
    free(label);
    free(cx);
    free(cy);
  } else {
    or_seed_population(L, K, NULL, NULL, NULL, NULL, NULL, N, 0, gp->seed, pop);
  }
}

void or_solve(const double* beta, int32_t L, int32_t K, const or_sinr_params* sp,
              const or_ga_params* gp, const int32_t* user_xy_mm, const int32_t* bs_xy_mm,
              int32_t kmeans_k, int32_t kmeans_max_iter, int32_t n_seeded, int32_t G,
              uint8_t* pop_out, double* fit_out, uint8_t* best_out, double* best_fit,
              double* hist_best) {
  const int32_t N = gp->N;
  const int64_t LK = (int64_t)L * K;
  uint8_t* pop = (uint8_t*)malloc((size_t)(N * LK));
  uint8_t* nxt = (uint8_t*)malloc((size_t)(N * LK));
  double* fit = (double*)malloc(sizeof(double) * (size_t)N);
  initial_population(L, K, gp, user_xy_mm, bs_xy_mm, kmeans_k, kmeans_max_iter, n_seeded, pop);
  for (int32_t g = 0; g < G; ++g) {
    or_fitness_batch(beta, L, K, pop, N, sp, fit);
    if (hist_best) hist_best[g] = fit[argbest(fit, N)];
    or_ga_step(pop, fit, L, K, gp, g, nxt);
    uint8_t* t = pop;
    pop = nxt;
    nxt = t;
  }
  or_fitness_batch(beta, L, K, pop, N, sp, fit);
  int32_t b = argbest(fit, N);
  if (hist_best) hist_best[G] = fit[b];
  if (pop_out) memcpy(pop_out, pop, (size_t)(N * LK));
  if (fit_out) memcpy(fit_out, fit, sizeof(double) * (size_t)N);
  if (best_out) memcpy(best_out, pop + b * LK, (size_t)LK);
  if (best_fit) *best_fit = fit[b];
  free(pop);
  free(nxt);
  free(fit);
}

/* ------------------------------------------------------------------------ */
/* PK-means GA (Sec. 4.3, Alg. 2): the population is partitioned by K-means */
/* and every cluster (island) evolves on its own; K-means is re-applied     */
/* every R generations (Sec. 6.1: every three).                             */
/* ------------------------------------------------------------------------ */

/* Chromosome n as one-hot pilot indicators e(n)[u][p] = (X_n[u] == p), one
 * K-vector per user u = l*K + k.  Centroid c of m_c members has per-user
 * pilot counts cnt_c[u][p] (centroid = cnt_c / m_c).  Then
 *   m_c^2 * ||e(n) - cnt_c/m_c||^2 = LK m_c^2 - 2 m_c S(n,c) + Q_c,
 *   S(n,c) = sum_u cnt_c[u][X_n[u]],   Q_c = sum_u sum_p cnt_c[u][p]^2,
 * an integer; two distances compare exactly by cross-multiplying with the
 * other cluster's m^2 (every factor below 2^37 when N, LK <= 4096, so every
 * product fits in 63 bits). */
static int64_t scaled_dist(const int64_t* cnt_c, int64_t m_c, int64_t q_c, const uint8_t* X,
                           int32_t LK, int32_t K) {
  int64_t S = 0;
  for (int32_t u = 0; u < LK; ++u) S += cnt_c[(int64_t)u * K + X[u]];
  return (int64_t)LK * m_c * m_c - 2 * m_c * S + q_c;
}

int32_t or_pop_kmeans(const uint8_t* pop, int32_t N, int32_t L, int32_t K, int32_t C,
                      int32_t max_iter, uint64_t seed, int32_t gen, int32_t* label,
                      int32_t* init_out) {
  const int32_t LK = L * K;
  const int64_t csz = (int64_t)LK * K;
  int64_t* cnt = (int64_t*)calloc((size_t)(C * csz), sizeof(int64_t));
  int64_t* ncnt = (int64_t*)calloc((size_t)(C * csz), sizeof(int64_t));
  int64_t* m = (int64_t*)calloc((size_t)C, sizeof(int64_t));
  int64_t* nm = (int64_t*)calloc((size_t)C, sizeof(int64_t));
  int64_t* q = (int64_t*)calloc((size_t)C, sizeof(int64_t));
  /* initial centroids: C distinct members by a partial Fisher-Yates shuffle */
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  for (int32_t i = 0; i < N; ++i) idx[i] = i;
  for (int32_t c = 0; c < C; ++c) {
    int32_t j = c + (int32_t)below(or_draw32(seed, 0, (uint64_t)gen, TAG_ISLAND, (uint32_t)c),
                                   (uint32_t)(N - c));
    int32_t t = idx[c];
    idx[c] = idx[j];
    idx[j] = t;
    const uint8_t* X = pop + (int64_t)idx[c] * LK;
    for (int32_t u = 0; u < LK; ++u) cnt[c * csz + (int64_t)u * K + X[u]] = 1;
    m[c] = 1;
    if (init_out) init_out[c] = idx[c];
  }
  free(idx);
  for (int32_t n = 0; n < N; ++n) label[n] = -1;
  int32_t passes = 0;
  for (int32_t it = 0; it < max_iter; ++it) {
    for (int32_t c = 0; c < C; ++c) {
      q[c] = 0;
      for (int64_t i = 0; i < csz; ++i) q[c] += cnt[c * csz + i] * cnt[c * csz + i];
    }
    /* assignment: nearest centroid, ties to the lower cluster index */
    int64_t changed = 0;
    for (int32_t n = 0; n < N; ++n) {
      const uint8_t* X = pop + (int64_t)n * LK;
      int32_t best = 0;
      int64_t bd = scaled_dist(cnt, m[0], q[0], X, LK, K);
      for (int32_t c = 1; c < C; ++c) {
        int64_t d = scaled_dist(cnt + c * csz, m[c], q[c], X, LK, K);
        /* d / m_c^2 < bd / m_best^2 */
        if (d * m[best] * m[best] < bd * m[c] * m[c]) {
          bd = d;
          best = c;
        }
      }
      if (label[n] != best) changed++;
      label[n] = best;
    }
    passes++;
    if (changed == 0 || it == max_iter - 1) break;
    /* update: the members' counts; an empty cluster keeps its centroid */
    memset(ncnt, 0, sizeof(int64_t) * (size_t)(C * csz));
    memset(nm, 0, sizeof(int64_t) * (size_t)C);
    for (int32_t n = 0; n < N; ++n) {
      const uint8_t* X = pop + (int64_t)n * LK;
      for (int32_t u = 0; u < LK; ++u) ncnt[label[n] * csz + (int64_t)u * K + X[u]] += 1;
      nm[label[n]] += 1;
    }
    for (int32_t c = 0; c < C; ++c)
      if (nm[c] > 0) {
        memcpy(cnt + c * csz, ncnt + c * csz, sizeof(int64_t) * (size_t)csz);
        m[c] = nm[c];
      }
  }
  free(cnt);
  free(ncnt);
  free(m);
  free(nm);
  free(q);
  return passes;
}

/* Tournament among the m members of one island (member list mem). */
static int32_t island_tournament(const double* fit, const int32_t* mem, int32_t m, int32_t tour,
                                 uint64_t seed, int32_t slot, int32_t gen, uint32_t first) {
  int32_t best = mem[below(or_draw32(seed, slot, gen, TAG_GA, first), (uint32_t)m)];
  for (int32_t t = 1; t < tour; ++t) {
    int32_t c = mem[below(or_draw32(seed, slot, gen, TAG_GA, first + t), (uint32_t)m)];
    if (better(fit, c, best)) best = c;
  }
  return best;
}

/* Island c owns the slots of its members.  With min(E, m_c) elites per
 * island and the child draws of slot n exactly as in or_ga_step, one island
 * holding the whole population is the plain generation. */
void or_island_step(const uint8_t* pop, const double* fit, int32_t L, int32_t K,
                    const or_ga_params* gp, int32_t gen, const int32_t* label, int32_t C,
                    uint8_t* next) {
  const int32_t N = gp->N, T = gp->tour;
  const int64_t LK = (int64_t)L * K;
  int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  char* taken = (char*)malloc((size_t)N);
  for (int32_t c = 0; c < C; ++c) {
    int32_t m = 0;
    for (int32_t n = 0; n < N; ++n)
      if (label[n] == c) mem[m++] = n;
    if (m == 0) continue;
    const int32_t Ec = gp->E < m ? gp->E : m;
    /* the island's elites, best first, into its first slots */
    memset(taken, 0, (size_t)N);
    for (int32_t e = 0; e < Ec; ++e) {
      int32_t best = -1;
      for (int32_t i = 0; i < m; ++i)
        if (!taken[mem[i]] && (best < 0 || better(fit, mem[i], best))) best = mem[i];
      taken[best] = 1;
      memcpy(next + mem[e] * LK, pop + best * LK, (size_t)LK);
    }
    for (int32_t i = Ec; i < m; ++i) {
      const int32_t n = mem[i];
      uint8_t* child = next + n * LK;
      int32_t a = island_tournament(fit, mem, m, T, gp->seed, n, gen, 0);
      int32_t b = island_tournament(fit, mem, m, T, gp->seed, n, gen, (uint32_t)T);
      uint32_t u_cross = or_draw32(gp->seed, n, gen, TAG_GA, (uint32_t)(2 * T));
      uint32_t u_cut = or_draw32(gp->seed, n, gen, TAG_GA, (uint32_t)(2 * T + 1));
      int32_t cut = L;
      if ((uint64_t)u_cross < gp->pc_thresh) cut = 1 + (int32_t)below(u_cut, (uint32_t)(L - 1));
      for (int32_t l = 0; l < L; ++l) {
        const uint8_t* src = (l < cut) ? pop + a * LK : pop + b * LK;
        memcpy(child + l * K, src + l * K, (size_t)K);
      }
      for (int32_t l = 0; l < L; ++l) {
        uint32_t base = (uint32_t)(2 * T + 2 + 3 * l);
        uint32_t u_mut = or_draw32(gp->seed, n, gen, TAG_GA, base);
        uint32_t ui = or_draw32(gp->seed, n, gen, TAG_GA, base + 1);
        uint32_t uj = or_draw32(gp->seed, n, gen, TAG_GA, base + 2);
        if ((uint64_t)u_mut < gp->pm_thresh) swap_two(child + l * K, K, ui, uj);
      }
    }
  }
  free(mem);
  free(taken);
}

void or_solve_islands(const double* beta, int32_t L, int32_t K, const or_sinr_params* sp,
                      const or_ga_params* gp, const int32_t* user_xy_mm, const int32_t* bs_xy_mm,
                      int32_t kmeans_k, int32_t kmeans_max_iter, int32_t n_seeded, int32_t G,
                      int32_t C, int32_t R, int32_t iters, uint8_t* pop_out, double* fit_out,
                      uint8_t* best_out, double* best_fit, double* hist_best,
                      int32_t* label_out) {
  const int32_t N = gp->N;
  const int64_t LK = (int64_t)L * K;
  uint8_t* pop = (uint8_t*)malloc((size_t)(N * LK));
  uint8_t* nxt = (uint8_t*)malloc((size_t)(N * LK));
  double* fit = (double*)malloc(sizeof(double) * (size_t)N);
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  for (int32_t n = 0; n < N; ++n) label[n] = 0;
  initial_population(L, K, gp, user_xy_mm, bs_xy_mm, kmeans_k, kmeans_max_iter, n_seeded, pop);
  for (int32_t g = 0; g < G; ++g) {
    /* Alg. 2: apply K-means (every R generations) and compute fitness */
    or_fitness_batch(beta, L, K, pop, N, sp, fit);
    if (hist_best) hist_best[g] = fit[argbest(fit, N)];
    if (g % R == 0) or_pop_kmeans(pop, N, L, K, C, iters, gp->seed, g, label, NULL);
    /* every island evolves on its own slots; the union is the population */
    or_island_step(pop, fit, L, K, gp, g, label, C, nxt);
    uint8_t* t = pop;
    pop = nxt;
    nxt = t;
  }
  or_fitness_batch(beta, L, K, pop, N, sp, fit);
  int32_t b = argbest(fit, N);
  if (hist_best) hist_best[G] = fit[b];
  if (pop_out) memcpy(pop_out, pop, (size_t)(N * LK));
  if (fit_out) memcpy(fit_out, fit, sizeof(double) * (size_t)N);
  if (best_out) memcpy(best_out, pop + b * LK, (size_t)LK);
  if (best_fit) *best_fit = fit[b];
  if (label_out) memcpy(label_out, label, sizeof(int32_t) * (size_t)N);
  free(pop);
  free(nxt);
  free(fit);
  free(label);
}

/* ------------------------------------------------------------------------ */
/* Exhaustive search (EX-PA, Sec. 6.2; Table 3 O(K!^(L-1))).                 */
/* ------------------------------------------------------------------------ */

/* Next permutation in lexicographic order; returns 0 after the last one. */
static int next_perm(uint8_t* a, int32_t K) {
  int32_t i = K - 2;
  while (i >= 0 && a[i] >= a[i + 1]) i--;
  if (i < 0) return 0;
  int32_t j = K - 1;
  while (a[j] <= a[i]) j--;
  uint8_t t = a[i];
  a[i] = a[j];
  a[j] = t;
  for (int32_t x = i + 1, y = K - 1; x < y; ++x, --y) {
    t = a[x];
    a[x] = a[y];
    a[y] = t;
  }
  return 1;
}

double or_exhaustive(const double* beta, int32_t L, int32_t K, const or_sinr_params* sp,
                     int32_t all_rows, uint8_t* best_X, int64_t* n_evaluated) {
  const int64_t LK = (int64_t)L * K;
  uint8_t* X = (uint8_t*)malloc((size_t)LK);
  for (int32_t l = 0; l < L; ++l)
    for (int32_t k = 0; k < K; ++k) X[l * K + k] = (uint8_t)k;
  const int32_t first_free = all_rows ? 0 : 1;
  double best = -INFINITY;
  int64_t count = 0;
  for (;;) {
    double f = or_fitness(beta, L, K, X, sp, NULL, NULL);
    count++;
    if (f > best) {
      best = f;
      if (best_X) memcpy(best_X, X, (size_t)LK);
    }
    /* odometer over rows L-1 .. first_free */
    int32_t l = L - 1;
    while (l >= first_free) {
      if (next_perm(X + l * K, K)) break;
      /* row wrapped to the last permutation: reset to identity, carry */
      for (int32_t k = 0; k < K; ++k) X[l * K + k] = (uint8_t)k;
      l--;
    }
    if (l < first_free) break;
  }
  free(X);
  if (n_evaluated) *n_evaluated = count;
  return best;
}
