/*
 * pa.h -- C ABI of the GB300 pilot-assignment library (libpa.so).
 *
 * Method: K-means-seeded two-dimensional genetic algorithm for uplink pilot
 * assignment in multi-cell massive MIMO (arXiv 2511.20511).  The data-
 * parallel hot path is the population-wide fitness evaluation (Sec. 3.2,
 * Eq. 3-6: per-user uplink SINR and spectral efficiency, summed over all
 * users); around it sit the GA generation step (Alg. 1: elitism, selection,
 * crossover, mutation) and the K-means population seeding (Sec. 1 item 2,
 * Alg. 1 "Apply K-means clustering").
 *
 * Conventions shared by every entry point
 *   beta[(j*L + l)*K + k]  large-scale fading (Eq. 2) of user k of cell l
 *                          at BS j; host memory, float64, finite and > 0.
 *   pop[(n*L + l)*K + k]   uint8 pilot of user k of cell l in chromosome n
 *                          (Sec. 4.1: one row per cell, each row a
 *                          permutation of 0..K-1).  Row-major, no padding.
 *   fitness                float32 (PA_FP32 contexts) or float64 (PA_FP64),
 *                          one value per chromosome: sum SE of Eq. 6, or
 *                          the smallest per-user SINR (PA_OBJ_MIN_SINR).
 *   "device" pointers      CUDA global memory on the context's device.
 *   "host" pointers        ordinary (pageable or pinned) host memory.
 *   Ownership              the caller owns every buffer it passes; the
 *                          context owns copies of beta and positions and
 *                          its resident population.
 *   Streams                work is enqueued on the context stream (given at
 *                          pa_create or pa_set_stream; NULL = legacy default
 *                          stream).  Calls marked "asynchronous" return
 *                          before the GPU finishes; the others synchronise
 *                          the context stream before returning.
 *   Errors                 no call aborts, exits or traps.  Invalid
 *                          arguments return PA_EINVAL before any GPU work;
 *                          CUDA failures return PA_ECUDA; pa_last_error()
 *                          then holds a message.  A context is not thread
 *                          safe; distinct contexts are independent.
 */
#ifndef PA_H
#define PA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pa_ctx pa_ctx;

typedef enum {
  PA_OK = 0,
  PA_EINVAL = 1,        /* invalid argument or configuration              */
  PA_ENOMEM = 2,        /* device or host allocation failed               */
  PA_ECUDA = 3,         /* a CUDA call failed (see pa_last_error)         */
  PA_ETIMEOUT = 4,      /* a bounded device wait gave up                  */
  PA_EUNSUPPORTED = 5,  /* valid but outside what the library implements */
  PA_EBUSY = 6          /* resource (slot, memory budget) not available   */
} pa_status;

/* Arithmetic of the fitness evaluation. */
enum {
  PA_FP32 = 0,  /* fast path: FP32 gathers and sums, <= 1e-5 relative     */
  PA_FP64 = 1   /* parity path: FP64, same operation order as the oracle  */
};

/* SINR model (Sec. 3.2). */
enum {
  PA_SINR_ASYMPTOTIC = 0, /* Eq. 4-5: beta_jjk^2 / sum_{l!=j} beta_jl(p)^2 */
  PA_SINR_FINITE_M = 1    /* Eq. 3 read with M antennas, MMSE pilot
                             estimates and MR combining:
                             M b^2 / (M S2 + (B_j + s2/rho)(S1 + s2/(tau_p rho))) */
};

/* Objective maximised by the GA. */
enum {
  PA_OBJ_SUM_SE = 0,  /* Eq. 7: sum over users of log2(1 + SINR) (Eq. 5-6)    */
  PA_OBJ_MIN_SINR = 1 /* Sec. 2: the smallest per-user SINR (max-min), with the
                         SINR of the chosen mode (not passed through log2)     */
};

/*
 * Configuration.  Fill with pa_config_default() and override fields.
 * Layout is fixed (128 bytes, natural alignment).
 */
typedef struct {
  int32_t L;        /* cells (>= 2)                                        */
  int32_t K;        /* users per cell = pilots per cell (1..64)            */
  int32_t tau_p;    /* pilot length (FINITE_M only; >= 1)                  */
  int32_t mode;     /* PA_SINR_*                                           */
  double M;         /* BS antennas (FINITE_M only; > 0)                    */
  double rho;       /* SNR scale: data/pilot power over noise unit (> 0)   */
  double sigma2;    /* noise variance (>= 0)                               */
  int32_t prec;     /* PA_FP32 or PA_FP64                                  */
  int32_t N;        /* population size (>= 2)                              */
  int32_t E;        /* elites copied unchanged (0 <= E < N)                */
  int32_t tour;     /* tournament size (>= 1)                              */
  uint64_t pc_thresh; /* crossover iff 32-bit draw < pc_thresh (0..2^32)   */
  uint64_t pm_thresh; /* per-row swap iff draw < pm_thresh (0..2^32)       */
  uint64_t seed;    /* Philox key of every random draw                     */
  int32_t kmeans_k; /* K-means clusters (1..K)                             */
  int32_t kmeans_max_iter; /* assignment passes (>= 1)                     */
  int32_t n_seeded; /* members built from the K-means assignment (0..N)   */
  int32_t flags;    /* 0, or PA_FLAG_TEST_STALL_COPIES                      */
  int32_t objective;   /* PA_OBJ_SUM_SE or PA_OBJ_MIN_SINR                  */
  int32_t islands;     /* 0 or 1: one population (Alg. 1); C in 2..64: the
                          PK-means GA of Alg. 2 with C islands (N <= 4096)  */
  int32_t recluster;   /* islands: generations between re-clusterings of
                          the population (>= 1; Sec. 6.1: every three)      */
  int32_t island_iter; /* islands: K-means passes per re-clustering (>= 1)  */
  int64_t reserved[2]; /* must be 0                                        */
} pa_config;

/*
 * Testing the bounded waits.  With this flag the context's next FP32
 * evaluation that stages chromosome tiles by bulk copies announces the
 * copies to its mbarriers but never issues them: every block's wait gives
 * up after about a second (the kernel returns normally, nothing faults),
 * and the next synchronous call reports PA_ETIMEOUT.  One-shot: later
 * evaluations of the context run normally.  The paper has no counterpart.
 */
#define PA_FLAG_TEST_STALL_COPIES 1

/*
 * Defaults for an L-cell, K-user layout: FP32, asymptotic SINR, sum-SE
 * objective (Eq. 7), tau_p = K, M = 256, rho = 10 / 500^-3.8 (10 dB at a
 * 500 m cell edge without shadowing), sigma2 = 1, N = 256, E = 2, tour = 3,
 * p_c = 0.9 (Table 1), p_m = 0.05 per row, seed 0, kmeans_k = K,
 * kmeans_max_iter = 100, n_seeded = (N + 1) / 2, islands = 0 (one
 * population), recluster = 3 and island_iter = 100 (used once islands >= 2).
 * Returns PA_EINVAL if cfg is NULL.
 */
pa_status pa_config_default(pa_config* cfg, int32_t L, int32_t K);

/* floor(p * 2^32) clamped to [0, 2^32]: threshold for a Bernoulli(p) draw. */
uint64_t pa_prob_to_thresh(double p);

/*
 * Create a context for one pilot-assignment instance on the current CUDA
 * device.  beta: host, L*L*K float64 (copied).  user_xy_mm (L*K*2) and
 * bs_xy_mm (L*2): host int32 positions in millimetres (copied), both NULL to
 * disable K-means seeding (random initial population instead).  stream:
 * cudaStream_t or NULL.  Prepares the per-instance tables on the GPU
 * (scaled gain tables, per-BS totals) and allocates the resident
 * population (2 * N * L * K bytes).  Synchronous.
 */
pa_status pa_create(const pa_config* cfg, const double* beta, const int32_t* user_xy_mm,
                    const int32_t* bs_xy_mm, void* stream, pa_ctx** out);

/*
 * Replace the instance of an existing context (same L, K and configuration):
 * beta (host, L*L*K float64) and optional positions as in pa_create.  The
 * gain tables are rebuilt on the GPU; the resident population is left as
 * it is and the generation counter reset to 0.  Asynchronous with respect
 * to the GPU work (the host arrays may be reused when the call returns
 * only if they are pageable; pinned arrays must stay untouched until the
 * context stream reaches this point).  PA_EINVAL on invalid values.
 */
pa_status pa_load_instance(pa_ctx* ctx, const double* beta, const int32_t* user_xy_mm,
                           const int32_t* bs_xy_mm);

/* Destroy a context and free its device memory (NULL is ignored). */
void pa_destroy(pa_ctx* ctx);

/* Replace the seed of every later random draw (seeding and GA steps). */
pa_status pa_set_seed(pa_ctx* ctx, uint64_t seed);

/* Replace the context stream (cudaStream_t or NULL). */
pa_status pa_set_stream(pa_ctx* ctx, void* stream);

/*
 * Fitness of n chromosomes (Eq. 6 sum SE with the per-user SINR of Eq. 4-5
 * or the finite-M reading of Eq. 3).  pop_dev: device, n*L*K bytes;
 * fit_dev: device, n float32 (PA_FP32) or float64 (PA_FP64).  Rows that are
 * not permutations give an unspecified value but never an out-of-bounds
 * access.  n == 0 is a no-op.  Asynchronous.  The FP32 kernels stage data
 * in shared memory with bulk copies under a bounded wait (about a second);
 * a wait that gives up leaves the outputs unspecified and is reported as
 * PA_ETIMEOUT by the context's next synchronous call
 * (pa_eval_population_host, pa_solve, pa_get_population).
 */
pa_status pa_eval_population(pa_ctx* ctx, const uint8_t* pop_dev, int64_t n, void* fit_dev);

/*
 * Same as pa_eval_population with host buffers: copies pop_host to the
 * device, evaluates, copies the fitness back.  Synchronous.
 */
pa_status pa_eval_population_host(pa_ctx* ctx, const uint8_t* pop_host, int64_t n,
                                  void* fit_host);

/*
 * One GA generation (Alg. 1: selection, crossover, mutation, with the
 * elitism of Sec. 1) from population pop_dev (device, N*L*K bytes) and its
 * fitness fit_dev (device, N values) into next_dev (device, N*L*K bytes,
 * must not overlap pop_dev).  Draws are Philox4x64-10 keyed by (seed,
 * child slot, generation).  Asynchronous.
 */
pa_status pa_ga_step(pa_ctx* ctx, const uint8_t* pop_dev, const void* fit_dev,
                     int32_t generation, uint8_t* next_dev);

/*
 * K-means on the users' positions relative to their own BS, then build the
 * resident population from the clustering (generation counter reset to 0).
 * Without positions, builds a random population.  labels_host (L*K int32)
 * and centroids_host (kmeans_k*2 float64, x then y per cluster) are
 * optional outputs; when either is given the call synchronises.
 */
pa_status pa_kmeans_seed(pa_ctx* ctx, int32_t* labels_host, double* centroids_host);

/*
 * Run `generations` GA generations on the resident population.  Async.
 * With cfg.islands = C >= 2 every generation is one of Alg. 2: before the
 * generations whose counter is a multiple of cfg.recluster (and before the
 * first one after seeding, pa_set_population or pa_load_instance) the
 * population is re-clustered into C islands (pa_island_cluster), then each
 * island evolves on its own slots (pa_island_step).
 */
pa_status pa_step(pa_ctx* ctx, int32_t generations);

/*
 * Whole solve (Alg. 1, or Alg. 2 with cfg.islands >= 2): seed
 * (pa_kmeans_seed), `generations` generations, final evaluation, best member
 * by (fitness desc, index asc).  best_host: L*K bytes; best_fit: its
 * fitness.  Synchronous.
 */
pa_status pa_solve(pa_ctx* ctx, int32_t generations, uint8_t* best_host, double* best_fit);

/*
 * Copy the resident population (N*L*K bytes) and optionally its fitness
 * (N values, evaluated now) and generation counter to the host.  Sync.
 */
pa_status pa_get_population(pa_ctx* ctx, uint8_t* pop_host, void* fit_host,
                            int32_t* generation);

/* Load a population (host, N*L*K bytes, rows must be permutations) and a
 * generation counter: checkpoint resume.  Synchronous; PA_EINVAL on an
 * invalid row. */
pa_status pa_set_population(pa_ctx* ctx, const uint8_t* pop_host, int32_t generation);

/* Device pointers of the resident population and its fitness buffer. */
pa_status pa_population_device(pa_ctx* ctx, uint8_t** pop_dev, void** fit_dev);

/* ------------------------------------------------------------------------
 * PK-means GA (Sec. 4.3, Alg. 2): the population is partitioned by K-means
 * into C = cfg.islands clusters ("islands") that evolve independently.  A
 * chromosome is represented by its one-hot pilot indicators (one K-vector
 * per user): the squared distance of two chromosomes is twice the number of
 * users whose pilots differ, and a centroid holds each user's pilot
 * frequencies over the cluster's members.  Distances are compared exactly
 * in integer arithmetic.  Requires a context created with islands >= 2.
 * ------------------------------------------------------------------------ */

/*
 * K-means of the N chromosomes of pop_dev (device, N*L*K bytes) into
 * cfg.islands clusters: initial centroids are distinct members drawn by a
 * partial Fisher-Yates shuffle keyed by (seed, generation); at most
 * cfg.island_iter Lloyd passes; ties go to the lower cluster; an emptied
 * cluster keeps its centroid.  labels_dev: device, N int32 (cluster of each
 * member).  passes_host (optional): the number of assignment passes; when
 * given the call synchronises, otherwise it is asynchronous.  Rows are
 * expected to be permutations; a pilot >= K is read as K-1.
 */
pa_status pa_island_cluster(pa_ctx* ctx, const uint8_t* pop_dev, int32_t generation,
                            int32_t* labels_dev, int32_t* passes_host);

/*
 * One generation of Alg. 2 from population pop_dev and its fitness fit_dev
 * (device, N values) with the clustering labels_dev (device, N int32 in
 * 0..C-1; other values are clamped into that range) into next_dev (device,
 * must not overlap pop_dev).  Island c owns the slots of its members: its
 * min(E, m_c) best members (fitness desc, index asc) go unchanged to its
 * lowest slots, every other slot gets a child of two tournaments among the
 * island's members, crossover and mutation with the draws pa_ga_step uses
 * for that slot -- so a single island is exactly pa_ga_step.  Asynchronous.
 */
pa_status pa_island_step(pa_ctx* ctx, const uint8_t* pop_dev, const void* fit_dev,
                         const int32_t* labels_dev, int32_t generation, uint8_t* next_dev);

/*
 * Island of every member of the resident population (host, N int32), from
 * the last re-clustering of pa_step / pa_solve (all -1 before the first).
 * Synchronous.
 */
pa_status pa_get_islands(pa_ctx* ctx, int32_t* labels_host);

/*
 * Check that every row of n chromosomes (device) is a permutation of
 * 0..K-1.  *first_bad = index of the first bad chromosome or -1.  Sync.
 */
pa_status pa_validate_population(pa_ctx* ctx, const uint8_t* pop_dev, int64_t n,
                                 int64_t* first_bad);

/* ------------------------------------------------------------------------
 * Batches: many independent instances, possibly of different L, K and N,
 * solved together.  Instances sharing a kernel variant (precision, SINR mode,
 * L rounded up to a multiple of 4, K <= 16 or not) run as one persistent
 * launch in which thread-block clusters take instances from a queue; the
 * seeding of all instances is one launch; the whole batch solve is captured
 * once per generation count into a CUDA graph and replayed.  Each instance
 * gives exactly the result pa_solve gives for it alone.
 * ------------------------------------------------------------------------ */
typedef struct pa_batch pa_batch;

/*
 * Create a batch of n instances: cfgs[i], betas[i] (host, L_i*L_i*K_i
 * float64) and optional positions user_xy_mm[i] / bs_xy_mm[i] as for
 * pa_create (the arrays of positions may be NULL for all instances).  Work
 * goes to `stream` (NULL: a stream the batch creates; the legacy default
 * stream cannot be captured into a graph).  Synchronous.  On failure
 * pa_last_error(NULL) explains.
 */
pa_status pa_batch_create(int32_t n, const pa_config* cfgs, const double* const* betas,
                          const int32_t* const* user_xy_mm, const int32_t* const* bs_xy_mm,
                          void* stream, pa_batch** out);

/* Destroy a batch and all its device memory (NULL is ignored). */
void pa_batch_destroy(pa_batch* b);

/* Replace instance i's gains and positions (same shapes; positions exactly
 * when the instance was created with them).  Asynchronous. */
pa_status pa_batch_load(pa_batch* b, int32_t i, const double* beta, const int32_t* user_xy_mm,
                        const int32_t* bs_xy_mm);

/*
 * Autotune the tiling: for each kernel-variant group, time the group's
 * solve for `generations` generations on the batch itself with every shape
 * that fits -- CTAs of 1024 threads (one CTA per SM; each evaluation thread
 * takes up to five column pairs, or up to two as the one-instance solve
 * does: the latency split) or of 256 threads (four per SM, so several
 * instances share an SM), in clusters of 1, 2, 4, 8 or 16 CTAs per
 * instance -- and keep the fastest, judged by the whole batch's time (the
 * groups run concurrently); then, per group, how many of its persistent
 * clusters may be resident at once (all that fit, or 7/8 down to 1/2 of
 * that, leaving SMs to the groups running beside it).  chosen (optional,
 * one entry per group) receives the chosen cluster sizes (pa_batch_groups
 * gives the rest).  Runs real solves (results are discarded).  Synchronous.
 */
pa_status pa_batch_tune(pa_batch* b, int32_t generations, int32_t* chosen);

/* Number of kernel-variant groups, their cluster sizes, CTA sizes
 * (threads), column splits (1: the latency split) and persistent clusters
 * launched, and the group of each instance (each output optional). */
pa_status pa_batch_groups(pa_batch* b, int32_t* n_groups, int32_t* cluster_sizes,
                          int32_t* cta_threads, int32_t* latency_split,
                          int32_t* resident_clusters, int32_t* group_of_instance);

/*
 * Solve every instance (Alg. 1 as in pa_solve): best_host receives the best
 * members back to back (instance i at offset sum_{m<i} L_m*K_m bytes),
 * best_fit their fitness (n values).  Either may be NULL.  Synchronous.
 */
pa_status pa_batch_solve(pa_batch* b, int32_t generations, uint8_t* best_host, double* best_fit);

/*
 * Latency of each instance in the last pa_batch_solve: ms_host[i] = time
 * from the start of that solve's GPU work until instance i's best member
 * and final population were complete (device clock, %globaltimer).  The
 * instances of a batch are all submitted at once, so this is each one's
 * completion latency.  Synchronous.
 */
pa_status pa_batch_completion_times(pa_batch* b, double* ms_host);

/* Context of instance i (owned by the batch): for pa_get_population etc. */
pa_status pa_batch_context(pa_batch* b, int32_t i, pa_ctx** out);

/* Last error message of a batch ("" if none). */
const char* pa_batch_last_error(const pa_batch* b);

/* ------------------------------------------------------------------------
 * Continuous-batching server.  Requests (one instance each) are queued by
 * pa_server_submit.  Each pa_server_poll (1) collects the ticks the GPU has
 * finished, without waiting: their slots advance, and requests that reached
 * `generations` are queued as completions; (2) admits queued requests, in
 * arrival order, into resident slots of their (L, K) class while the device
 * memory of the slots stays within the budget (idle slots of other classes
 * are destroyed when the next request needs their memory); (3) launches one
 * tick for every active slot that has none in flight: the newly admitted
 * slots are seeded (one launch) and every slot of the tick advances by up
 * to `tick` generations (one persistent launch per kernel variant;
 * populations stay resident between ticks); (4) returns completions.  Up
 * to four ticks are in flight at once on streams of their own, so a request
 * admitted while another tick runs starts at once on the SMs it leaves
 * free.  pa_server_wait blocks until a tick finishes.  A request's result
 * equals pa_solve's for the same instance, configuration and seed.  A
 * request whose admission fails (its slot cannot be created or loaded)
 * completes with that status; the others are not affected.  Not thread
 * safe.
 * ------------------------------------------------------------------------ */
typedef struct pa_server pa_server;

/* Create a server: base supplies every configuration field except L, K,
 * tau_p and kmeans_k (set from each request: tau_p = kmeans_k = K) and seed
 * (per request).  budget_bytes bounds the device memory of all slots.
 * stream: cudaStream_t or NULL (a stream of its own).  PA_EINVAL for an
 * invalid base; PA_EUNSUPPORTED for islands >= 2 (islands run per
 * generation, outside the batched solve kernel). */
pa_status pa_server_create(const pa_config* base, int32_t generations, int32_t tick,
                           uint64_t budget_bytes, void* stream, pa_server** out);

/* Destroy a server and its slots (NULL is ignored). */
void pa_server_destroy(pa_server* s);

/*
 * Queue a request: beta (L*L*K float64, finite and > 0), user_xy_mm (L*K*2),
 * bs_xy_mm (L*2) host arrays, copied before returning; id is returned on
 * completion.  Checked here, before anything is queued: PA_EINVAL for an
 * invalid shape or invalid values (as pa_create would reject them),
 * PA_EUNSUPPORTED for a shape the batched solve kernel cannot run, PA_EBUSY
 * when one slot of this shape alone needs more device memory than the
 * budget.  PA_ENOMEM if the host copy cannot be made.
 */
pa_status pa_server_submit(pa_server* s, int64_t id, int32_t L, int32_t K, uint64_t seed,
                           const double* beta, const int32_t* user_xy_mm,
                           const int32_t* bs_xy_mm);

/*
 * One scheduling round (collect finished ticks, admit, launch; it does not
 * wait for the GPU), then up to max_done completions are returned in
 * completion order (the rest wait for later polls): done_ids[i],
 * done_status[i] (PA_OK, or why the request failed), their best member at
 * done_best + i*best_stride (L*K bytes; zeros for a failed request) and its
 * fitness done_fit[i] (NaN for a failed request) -- each output optional;
 * *n_done = how many.  n_active / n_pending (optional): slots still running
 * and requests still queued after the tick.  An error status means the tick
 * itself failed (a CUDA error): completions already queued stay queued.
 */
pa_status pa_server_poll(pa_server* s, int32_t max_done, int64_t* done_ids, int32_t* done_status,
                         uint8_t* done_best, int64_t best_stride, double* done_fit,
                         int32_t* n_done, int32_t* n_active, int32_t* n_pending);

/*
 * Block until the oldest tick in flight has finished (timeout_us < 0), or
 * at most timeout_us microseconds; returns at once when none is in flight.
 * The next pa_server_poll collects what finished.
 */
pa_status pa_server_wait(pa_server* s, int32_t timeout_us);

/*
 * Withdraw request `id`: removed from the queue, or its slot released (the
 * slot stays resident for the next request of its class; when a tick of it
 * is in flight, once that tick has finished, and its result is dropped), or
 * its unreturned completion dropped.  PA_EINVAL when no queued, running or
 * unreturned request has this id.
 */
pa_status pa_server_cancel(pa_server* s, int64_t id);

/* Device bytes held by slots, number of slots, requests completed (with or
 * without an error). */
pa_status pa_server_stats(const pa_server* s, uint64_t* used_bytes, int32_t* n_slots,
                          int64_t* completed);

/*
 * Testing the admission failure path without a device fault: the next
 * `count` admissions fail as if their slot could not be created (status
 * PA_ECUDA, nothing runs on the GPU for them).  The paper has no
 * counterpart.
 */
pa_status pa_server_inject_admission_failures(pa_server* s, int32_t count);

/* Last error message of a server ("" if none). */
const char* pa_server_last_error(const pa_server* s);

/*
 * Size of the device array behind pa_eval_population_noalloc (bytes).
 */
#define PA_NOALLOC_SCRATCH_BYTES (256u * 1024u)

/*
 * Fitness evaluation that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * a real-time scheduling loop that must not take cudaMalloc's implicit
 * device-wide synchronisation and unbounded latency, or a framework that
 * hands out all device memory from its own pool.  It computes exactly what
 * pa_create + pa_eval_population + pa_destroy compute for the same cfg and
 * beta, without a context: the instance copy and the prepared tables go to a
 * file-scope device array of PA_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * holds from library load to process exit.
 *   cfg      configuration: must pass the same validation as for pa_create
 *            (every field, the GA ones included); the instance, SINR and
 *            objective fields and prec (the fitness type) are the ones used
 *   beta     host, L*L*K float64 gains (as for pa_create)
 *   pop_dev  device, n*L*K bytes;  fit_dev  device, n float32 / float64
 *   stream   cudaStream_t or NULL
 * Instances needing more scratch than the array holds (gains + prepared
 * tables) return PA_EUNSUPPORTED; pa_last_error(NULL) says how much was
 * needed.  Invalid arguments return PA_EINVAL.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) for that device;
 * make that first call before any stream capture.  All calls share the array
 * and leave their data in it; each call rewrites what it reads, but calls
 * whose GPU work overlaps (unordered streams, concurrent host threads on one
 * device) race and give undefined results.  Copies beta from host memory and
 * synchronises the stream before returning.
 */
pa_status pa_eval_population_noalloc(const pa_config* cfg, const double* beta,
                                     const uint8_t* pop_dev, int64_t n, void* fit_dev,
                                     void* stream);

/* Static description of a status code. */
const char* pa_status_str(pa_status s);

/* Last error message of a context ("" if none).  With ctx == NULL: the
 * reason for the calling thread's last failed pa_create, pa_batch_create,
 * pa_server_create or pa_eval_population_noalloc (each of these clears it
 * when it starts). */
const char* pa_last_error(const pa_ctx* ctx);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts, all devices); for accounting launches in a timed region. */
uint64_t pa_kernel_launches(void);

/*
 * CTAs per thread-block cluster of the context's fused solve kernel (all
 * generations in one launch, one cluster per instance): *ctas = 1..16, 0
 * when the instance runs one evaluation and one GA launch per generation,
 * -1 before the first pa_solve / pa_step has chosen.  No GPU work.
 */
pa_status pa_solve_cluster_ctas(const pa_ctx* ctx, int32_t* ctas);

#ifdef __cplusplus
}
#endif
#endif /* PA_H */
