/*
 * ccm.h -- C ABI of the GB300-native convergent cross mapping (CCM) library.
 *
 * What one call computes (paper Sect. 1, Sect. 2.1, Sect. 3.1, Sect. 3.2; the
 * equations are the method's, as the paper takes them from Sugihara et al.
 * 2012):
 *
 *   For every pair (j, i) = (library variable, target variable), embedding
 *   dimension E, delay tau, library size L and realization k:
 *     - shadow manifold of series j: M_j(m) = (s_j[t], s_j[t-tau], ...,
 *       s_j[t-(E-1)tau]), t = m + (E-1)tau, m in [0, N_m), N_m = N-(E-1)tau
 *       (Sect. 1: lagged embedding; Sect. 3.2: "lagged-coordinate vector");
 *     - a random library of L distinct manifold points (Sect. 1: r random
 *       subsamples of size L; Sect. 3.1).  Point m is chosen when its key
 *       (v << 32 | m) is among the L smallest, v being 32-bit half number
 *       m mod 8 (hi(w0), lo(w0), hi(w1), ..., lo(w3)) of the block
 *       Philox4x64-10(ctr=(floor(m/8), k, L, (j<<16)|(E<<8)|tau),
 *       key=(seed, 0));
 *     - for every manifold point m (all N_m points are queries) its E+1
 *       nearest library points, m itself excluded (optionally every l with
 *       |l - m| <= W, ccm_problem.theiler), ordered by (squared FP32
 *       distance, manifold index) (Sect. 3.2);
 *     - simplex projection (Sect. 2.1): d_i the distances, u_i =
 *       exp(-d_i/d_1) (the limit 1 for d_i = 0, else 0, when d_1 = 0),
 *       optionally raised to a floor f (ccm_problem.weight_floor),
 *       w_i = u_i / sum u, Xhat(m) = sum_i w_i s_i[t_i];
 *     - the skill rho = Pearson(s_i[t_m], Xhat(m)) over m (Sect. 2.1),
 *       accumulated in FP64; NaN when either variance is zero.
 *
 * Precision: distances, selection, weights and predictions in FP32;
 * rho moments in FP64.
 *
 * Output layout: rho[pair][E][tau][L][k], FP64, C order, where the axes index
 * the arrays of ccm_problem in the order given.
 *
 * Ownership: the caller owns every buffer it passes.  A context owns the
 * device memory of its plans; a plan copies the problem description at
 * ccm_plan time, so the caller may free the ccm_problem arrays on return.
 * No exception crosses this ABI; every entry point returns a ccm_status, and
 * ccm_last_error() gives a thread-local message for the last failure.
 *
 * Threads: one context may be used from several host threads; a plan must
 * not be run concurrently with itself.
 */
#ifndef CCM_GB300_H
#define CCM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CCM_OK = 0,
  CCM_PENDING = 1,        /* ccm_poll: the job has not finished yet */
  CCM_EINVAL = -1,        /* invalid argument; nothing was run */
  CCM_ENOMEM = -2,        /* device or host allocation failed */
  CCM_ETOOLARGE = -3,     /* the job's device footprint exceeds the context budget */
  CCM_ECUDA = -4,         /* a CUDA call failed; see ccm_last_error() */
  CCM_ETIMEOUT = -5,      /* a bounded wait ran out */
  CCM_ECANCELLED = -6,    /* the job was cancelled */
  CCM_ENOTFOUND = -7      /* unknown ticket */
} ccm_status;

/* ccm_problem.flags */
#define CCM_INPUT_ON_DEVICE  0x1u  /* series pointers given to ccm_run are device memory */
#define CCM_OUTPUT_ON_DEVICE 0x2u  /* rho (and debug outputs) given to ccm_run are device memory */
#define CCM_NO_AUTOTUNE      0x4u  /* keep cached or default kernel parameters (see ccm_run) */
#define CCM_NO_TABLE         0x10u /* brute-force search for every realization: no distance
                                      indexing tables (paper Sect. 3.2).  By default,
                                      realizations with large L read their neighbours from
                                      per-(variable, E, tau) tables built in the same run,
                                      where that is faster and the tables fit a quarter of
                                      the context budget; results are identical either way.
                                      Tuning knobs (environment, read at each ccm_plan):
                                      CCM_TABLE_CROSSOVER (default 20), CCM_TABLE_FLOOR
                                      (default 256) and CCM_TABLE_MAX_RATIO (default 40):
                                      tables for L >= max(floor, sqrt(c*N_m/(E+1)),
                                      N_m/max_ratio); CCM_TABLE_SAFETY (default 1): factor
                                      on the table row length */
#define CCM_SEARCH_STATS     0x20u /* the neighbour-search kernels also count their work
                                      (ccm_plan_search_stats); a separately compiled
                                      counting variant, slower, same results */

typedef struct {
  int32_t n_series;        /* V >= 2 series, each of length n */
  int64_t n;               /* series length N */
  int32_t n_pairs;         /* number of (j, i) pairs */
  const int32_t* pairs;    /* [n_pairs][2] = (library var j, target var i), 0 <= i, j < V, i != j;
                              (pairs sharing a j) x ceil(n/256) must stay below 2^31 */
  int32_t n_E;
  const int32_t* E;        /* [n_E], each 1..10 */
  int32_t n_tau;
  const int32_t* tau;      /* [n_tau], each >= 1, with N_m = n - (E-1)tau >= E+2 */
  int32_t n_L;
  const int64_t* L;        /* [n_L], each E+2 <= L <= N_m for every (E, tau) of the grid */
  int32_t r;               /* realizations per (pair, E, tau, L) cell, >= 1 */
  uint64_t seed;           /* library sampler seed */
  uint32_t flags;          /* CCM_INPUT_ON_DEVICE | CCM_OUTPUT_ON_DEVICE | CCM_NO_AUTOTUNE |
                              CCM_NO_TABLE | CCM_SEARCH_STATS; other bits are refused
                              (CCM_EINVAL) */
  /* Two options the paper does not discuss (common CCM variants); zero for the
   * paper's method.  theiler: exclusion window W >= 0, library point l is a
   * neighbour candidate of query m only when |l - m| > W (W = 0 excludes m
   * itself, the paper's rule); needs L >= E + 2 + 2W for every cell.
   * weight_floor: f >= 0, finite; u_i = max(exp(-d_i/d_1), f) before the
   * weights are normalised (f is applied in FP32). */
  int32_t theiler;
  float weight_floor;
} ccm_problem;

/* Optional per-unit outputs for checking (all device or all host, following
 * CCM_OUTPUT_ON_DEVICE).  Units are ordered like rho.  Sizes: libraries
 * sum over units of L int32; neighbours sum of N_m*(E+1) int32 (row m of a
 * unit holds the E+1 neighbours of query m, nearest first); predictions sum
 * of N_m float32.  ccm_plan_info gives the totals.  Any member may be NULL. */
typedef struct {
  int32_t* libraries;
  int32_t* neighbours;
  float* predictions;
} ccm_debug_out;

typedef struct {
  int64_t n_units;            /* realizations = n_pairs*n_E*n_tau*n_L*r */
  int64_t n_queries;          /* sum over units of N_m */
  int64_t library_entries;    /* sum over units of L */
  int64_t neighbour_entries;  /* sum over units of N_m*(E+1) */
  int64_t n_work_items;       /* (unit, query tile) items of the fused kernel */
  size_t device_bytes;        /* device footprint of the plan */
  double pair_count;          /* query-library pairs = sum over units of N_m*L */
  double flop_count;          /* 3E FP32 flops per pair, summed */
  double brute_flop_count;    /* the part of flop_count searched by brute force */
  size_t table_bytes;         /* distance indexing tables of the plan (0: none) */
  int64_t launches_per_run;   /* kernel launches of one ccm_run (graph nodes) */
  double brute_pair_count;    /* the part of pair_count searched by brute force */
  int64_t search_query_count; /* neighbour searches: N_m summed over library realizations
                                 (a library realization serves all targets of its variable) */
  int64_t table_query_count;  /* the part of search_query_count answered from a distance
                                 indexing table; the rest are searched by brute force */
} ccm_plan_info;

typedef struct ccm_context ccm_context;
typedef struct ccm_plan_s ccm_plan_t;

/* Create a context on CUDA device `device` whose plans may hold at most
 * `hbm_budget_bytes` of device memory in total (0 = 90% of the free memory at
 * creation).  Starts the serving thread lazily on the first ccm_submit. */
ccm_status ccm_context_create(int device, size_t hbm_budget_bytes, ccm_context** out);

/* Cancel pending jobs, join the serving thread, free every plan's memory. */
ccm_status ccm_context_destroy(ccm_context* ctx);

/* Validate the problem, build the work list (units sorted by cost, split into
 * query tiles), reserve device memory.  Returns CCM_EINVAL for an invalid
 * problem and CCM_ETOOLARGE when the footprint exceeds the context budget. */
ccm_status ccm_plan(ccm_context* ctx, const ccm_problem* prob, ccm_plan_t** out);

ccm_status ccm_plan_destroy(ccm_plan_t* plan);

ccm_status ccm_plan_get_info(const ccm_plan_t* plan, ccm_plan_info* info);

/* Run the whole sweep: query order, observed-value tile moments (the target's
 * mean and centred values per query tile of each (pair, E, tau), shared by
 * every L and realization), distance indexing tables (unless
 * CCM_NO_TABLE or none pays off), library sampler, one persistent fused
 * kNN + simplex + rho kernel per E for the brute-force realizations and one
 * table-scan kernel for the rest; replayed from a CUDA graph after the first
 * call.
 * series: [n_series][n] FP32 (host unless CCM_INPUT_ON_DEVICE); rho: FP64 as
 * above (host unless CCM_OUTPUT_ON_DEVICE).  cuda_stream: a cudaStream_t, or
 * NULL to run on the plan's own stream and block until done.  With a caller
 * stream and device output the call is asynchronous; with host input or
 * output it synchronises the stream before returning.  Host series are
 * checked for non-finite values (CCM_EINVAL).
 * Autotuning: on the first ccm_run of a plan with at least 2e11 query-library
 * pairs, for every E whose parameters are not yet known to the context, the
 * library times two kernel variants and three merge triggers on a sample of
 * the plan's work items and keeps the fastest (results are identical for all
 * of them).  Choices are cached per (device name, E) in $CCM_AUTOTUNE_CACHE,
 * default ~/.cache/ccm_gb300/autotune.tsv, and loaded by ccm_context_create.
 * CCM_NO_AUTOTUNE skips the measurement. */
ccm_status ccm_run(ccm_plan_t* plan, const float* series, double* rho, void* cuda_stream);

/* ccm_run plus optional per-unit outputs (dbg may be NULL). */
ccm_status ccm_run_ex(ccm_plan_t* plan, const float* series, double* rho,
                      const ccm_debug_out* dbg, void* cuda_stream);

/* Device time of the preparation launches (query order, observed moments,
 * tables, sampler) and of the neighbour-search launches (brute force + table
 * scan) in the plan's last completed ccm_run / ccm_run_ex (CUDA events
 * recorded on the run's stream around each launch).  Call after that run has
 * finished. */
ccm_status ccm_plan_kernel_times(const ccm_plan_t* plan, double* sampler_ms, double* knn_ms);

/* The same events per stage: stage_ms[0] query order + observed-value tile
 * moments + distance indexing tables, [1] library sampler, [2] brute-force fused kernel, [3] table-scan
 * fused kernel (0 when the stage launched nothing). */
ccm_status ccm_plan_stage_times(const ccm_plan_t* plan, double* stage_ms /* [4] */);

/* Work counts of the neighbour search in the plan's last completed run
 * (plans made with CCM_SEARCH_STATS only; CCM_EINVAL otherwise).  They say how
 * much of the method's exhaustive work (N_m*L pairs per realization) the
 * brute-force kernels executed and what the selection cost.  Call after the
 * run has finished. */
typedef struct {
  uint64_t brute_tiles;      /* query tiles (256 queries) searched by brute force */
  uint64_t brute_queries;    /* their valid queries */
  uint64_t pairs_begun;      /* query-library pairs whose squared distance was begun (the
                                first coordinates of a step, before early termination) */
  uint64_t pairs_full;       /* pairs whose squared distance was completed (all E) */
  uint64_t pairs_pruned;     /* pairs skipped whole by the chunk bounding-box test */
  uint64_t candidates;       /* pairs below a query's running threshold, queued for insertion */
  uint64_t merge_slots;      /* insertion slots executed: per warp merge, 32 x the largest
                                queue of its lanes (lanes with shorter queues idle) */
  uint64_t table_queries;    /* queries answered from a distance indexing table */
  uint64_t table_entries;    /* table entries loaded by those queries' walks */
  uint64_t table_fallbacks;  /* of them, queries that met too few library members in their
                                row and scanned their library instead */
} ccm_search_stats;
ccm_status ccm_plan_search_stats(const ccm_plan_t* plan, ccm_search_stats* out);

/* The plain comparator: one sampler launch and one naive kNN launch per
 * realization (thread per query, library read from global memory, sorted
 * insertion), same precision and same results.  It exists to measure the
 * batched path against; rho/series placement as in ccm_run. */
ccm_status ccm_run_plain(ccm_plan_t* plan, const float* series, double* rho, void* cuda_stream);

/* Serving: queue a job (the context copies the series into pinned staging,
 * so the caller may free it on return).  The serving thread admits queued
 * jobs while their device footprints fit the free budget, batches admitted
 * jobs' work items into shared persistent launches, and overlaps them on
 * several streams.  CCM_ETOOLARGE if the footprint exceeds the whole budget.
 * A batch whose launch fails (a CUDA call returns an error) fails its own jobs
 * with CCM_ECUDA at ccm_poll; the other jobs and later batches are unaffected.
 * Test hook: the environment variable CCM_FAULT_INJECT_BATCH=n, read by
 * ccm_context_create, makes the launch of that context's batch n (0-based, in
 * launch order) fail on the host as if a CUDA call had failed after its
 * uploads were enqueued; no device work is faulted. */
ccm_status ccm_submit(ccm_context* ctx, const ccm_problem* prob, const float* series,
                      uint64_t* ticket);

/* Non-blocking when timeout_ms == 0, otherwise waits up to timeout_ms.
 * CCM_OK: rho (host, layout as ccm_run) written and the ticket retired;
 * CCM_PENDING: not done yet; CCM_ENOTFOUND: unknown or retired ticket;
 * a negative status if the job failed or was cancelled (ticket retired). */
ccm_status ccm_poll(ccm_context* ctx, uint64_t ticket, double* rho, int32_t timeout_ms);

/* Cancel a queued job that has not been admitted yet (CCM_PENDING if it is
 * already running; it then finishes normally). */
ccm_status ccm_cancel(ccm_context* ctx, uint64_t ticket);

/* Submit/admit/finish timestamps (seconds on the context's monotonic clock)
 * of a finished job that has not been polled yet. */
ccm_status ccm_job_times(ccm_context* ctx, uint64_t ticket, double* submit_s, double* start_s,
                         double* finish_s);

/* One CCM cell without any device allocation (the paper has no counterpart:
 * it exists for callers that cannot call cudaMalloc at run time, e.g. a host
 * framework whose own caching allocator owns the device memory, or a
 * latency-critical loop where cudaMalloc/cudaFree may synchronise the device).
 * Computes rho of pair (j, i), E, tau, L for realizations k = 0..r-1 with the
 * same sampler and fused kernel as ccm_run, so d_rho[k] equals the matching
 * entry of ccm_run's output for the same seed.
 * d_series: device [n_series][n] FP32 (not checked for non-finite values);
 * d_rho: device [r] FP64, written in stream order.  All scratch lives in one
 * fixed 16 MiB device array held by every GPU that loads the library until
 * exit; a cell needing more (about r*L*4 + r*ceil(N_m/256)*56 + r*160 +
 * N_m*4 + ceil(N_m/256)*2112 bytes) returns CCM_ETOOLARGE with a message and runs nothing.  Nothing is
 * allocated.  The first call on a device (with that device current) finds
 * the array's address and sets kernel attributes; make it before any stream
 * capture.  Every call reuses the same array: calls that overlap on the GPU
 * (several streams or host threads) race and must be serialised by the
 * caller.  cuda_stream NULL: runs on the default stream and blocks until done,
 * then reports kernel error flags (CCM_ECUDA).  Otherwise asynchronous, and
 * kernel error flags are NOT reported: the next call's set-up clears them, so
 * an asynchronous caller that needs the check must pass NULL. */
ccm_status ccm_run_noalloc(const float* d_series, int32_t n_series, int64_t n, int32_t j,
                           int32_t i, int32_t E, int32_t tau, int64_t L, int32_t r,
                           uint64_t seed, double* d_rho, void* cuda_stream);

/* Convergence decision for one (pair, E, tau) row of the rho grid. */
typedef struct {
  double rho_first;   /* mean rho of the finite realizations at the smallest L */
  double rho_last;    /* the same at the largest L */
  double jt;          /* Jonckheere-Terpstra J over the L groups in increasing L:
                         pairs (x earlier, y later) with y > x count 1, y == x 1/2 */
  double z;           /* (J - E[J]) / sqrt(Var[J]) with no trend, no tie correction:
                         E[J] = (N^2 - sum n_g^2)/4,
                         Var[J] = (N^2(2N+3) - sum n_g^2(2n_g+3))/72, N = sum n_g */
  int32_t n_valid;    /* finite realizations in the row (N) */
  int32_t converged;  /* 1 when z > z_crit, rho_last > rho_first and rho_last > 0 */
} ccm_convergence_t;

/* Convergence of cross-map skill with L (paper Sect. 1: skill should rise with
 * the library size, judged over the r realizations; the paper states no test,
 * this one-sided trend test is the reading taken).  rho: [n_rows][n_L][r] FP64,
 * the layout ccm_run writes (n_rows = n_pairs*n_E*n_tau); L: host [n_L], the
 * grid's library sizes in the order of rho's L axis (any order, distinct).
 * Non-finite rho are left out.  out: [n_rows].  flags: CCM_INPUT_ON_DEVICE
 * (rho is device memory), CCM_OUTPUT_ON_DEVICE (out is device memory); host
 * buffers are staged through temporary device memory.  Limits: 2 <= n_L <= 64,
 * n_L*r <= 24576.  cuda_stream as in ccm_run (NULL: blocks until done).
 * J is an exact integer and every FP64 step a round-to-nearest operation in a
 * fixed order (group means in realization order, sizes in increasing L), so
 * the result depends on nothing but the row. */
ccm_status ccm_convergence(ccm_context* ctx, const double* rho, int64_t n_rows, int32_t n_L,
                           const int64_t* L, int32_t r, double z_crit,
                           ccm_convergence_t* out, uint32_t flags, void* cuda_stream);

/* Thread-local message describing the last non-OK status on this thread. */
const char* ccm_last_error(void);

/* Library version string. */
const char* ccm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CCM_GB300_H */
