// Internal declarations shared by the CUDA kernels and the host runtime of the
// CCM library (not part of the public ABI, see include/ccm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ccm {

constexpr int kMaxE = 10;

// One library realization ("unit"): library variable j, E, tau, L, realization
// k of one job, with the targets it is cross-mapped to.  The library and the
// neighbour lists do not depend on the target, so all pairs (j, i) of a job
// that share j are computed from one neighbour search.
struct UnitDesc {
  int64_t series_off;   // element offset of the job's series block [V][n]
  int64_t n;            // series length of the job
  int64_t lib_off;      // offset of this unit's library in the library buffer
  int64_t part_off;     // first partial-moment slot: target t, tile q at part_off + t*n_tiles + q
  int64_t order_off;    // first entry of this unit's query order (per variable, E, tau)
  int64_t tgt_off;      // first TargetDesc of this unit
  int64_t table_off;    // distance indexing table of (j, E, tau), when table_R > 0
  uint64_t seed;        // library sampler seed of the job
  int32_t j;            // library variable
  int32_t E, tau;
  int32_t L, k;
  int32_t n_m;          // manifold points = queries
  int32_t n_tiles;      // query tiles of the fused kernel
  int32_t n_targets;    // targets cross-mapped from this library (>= 1)
  int32_t table_R;      // > 0: neighbours read from the table (R entries per query)
  int32_t theiler;      // exclusion window W >= 0: candidates l of query m need |l - m| > W
  float wfloor;         // simplex weight floor f >= 0: u_i = max(u_i, f)
  int32_t table_tv;     // 1: the table also holds this unit's (single) target's values
};

// One target of a unit: the pair (j, i) and where its outputs go.
struct TargetDesc {
  int64_t out_idx;      // index of this (pair, E, tau, L, k) in the rho buffer
  int64_t q_off;        // first query of this pair-realization in the debug predictions
  int64_t nbr_off;      // first entry in the debug neighbour lists
  int64_t lib_dbg_off;  // first entry in the debug libraries
  int64_t obs_tile;     // observed-moment record of query tile 0 of (j, i, E, tau)
  int32_t i;            // target variable
  int32_t pad;
};

// Observed-moment job: one per (job, library variable j, target i, E, tau).
// The observed values of a query tile (the target at the tile's manifold
// points) do not depend on L or the realization, so their tile mean, centred
// values and centred sum of squares are computed once per run and read by the
// epilogue of every realization of that (j, i, E, tau).
struct ObsJob {
  int64_t series_off;   // element offset of the job's series block
  int64_t n;            // series length
  int64_t order_off;    // query order of (j, E, tau)
  int64_t obs_tile;     // first tile record; the jobs' records are consecutive
  int32_t i, E, tau, n_m, n_tiles;
  int32_t pad;
};
// One tile record: x_q - mean(x) for the tile's 256 queries in query order
// (zero past the tile's end), then mean(x) and sum of (x_q - mean(x))^2.
constexpr int kObsStride = 264;        // doubles per record (64-byte multiple)

// One work item of the fused kernels: query tiles [tile, tile + chunk) of a
// unit (chunk = kBruteChunk for the brute-force kernel, kTableChunk for the
// table kernel; the last item of a unit may hold fewer tiles).
// A table item may cover `count` consecutive realizations of one cell (units
// unit .. unit + count - 1): one walk of each query's table row serves all of
// them.  Brute-force items have count 1.
struct WorkItem {
  int32_t unit;
  int32_t tile;
  int32_t count;
};
constexpr int kBruteChunk = 8;         // query tiles per brute-force work item (one staging)
constexpr int kTableGroup = 4;         // realizations per grouped table item, at most
constexpr int kTableGroupMaxNm = 32768;  // grouping needs a byte membership map (bit b: realization b)

// Query order job: one per (job, library variable, E, tau).
struct OrderJob {
  int64_t series_off;   // element offset of the job's series block
  int64_t n;            // series length
  int64_t order_off;    // first entry of the order array of this combination
  int64_t scratch_off;  // manifolds above kOrderMaxSort: 2*n_m 64-bit keys of scratch
                        // from here (merge sort); -1: keep time order
  int32_t j, E, tau, n_m;
};
constexpr int kOrderMaxSort = 16384;   // manifolds up to this size are sorted in one pass

// Distance indexing table job: one per (job, library variable, E, tau) whose
// realizations read their neighbours from a table.
struct TableJob {
  int64_t series_off;   // element offset of the job's series block
  int64_t n;            // series length
  int64_t order_off;    // query order of this combination
  int64_t table_off;    // first entry: table[table_off + r * n_m + pos]
  int32_t j, E, tau, n_m, R;
  int32_t tv_i;         // >= 0: also store target variable tv_i's value at every entry's point
};
constexpr int kTableMaxR = 2048;       // entries per query row, at most
constexpr int kTableChunk = 8;         // query tiles per table work item (one bitmap each)
constexpr int kTableMaxNm = 1 << 20;   // longest manifold that gets a table (bitmap in smem)

// Sampler: one CTA per unit.
struct SamplerParams {
  const UnitDesc* units;
  const TargetDesc* targets;  // for the debug copies (lib_dbg_off per target)
  const int32_t* order;   // query orders (per variable, E, tau); libraries follow them
  int32_t* lib;           // library buffer (sum of L), each library in query order
  int32_t* dbg_lib;       // optional: libraries in ascending m, once per target, in rho order
  int32_t* err;           // error flag (set, never cleared, by the kernels)
};

// Fused kNN + simplex + moments: persistent, one work item at a time.
struct KnnParams {
  const float* series;    // device series blocks
  const UnitDesc* units;
  const TargetDesc* targets;
  const WorkItem* items;
  int64_t n_items;
  const int32_t* lib;
  const int32_t* order;   // query order (manifold index per position)
  const void* table;      // distance indexing tables (units with table_R > 0)
  const float* table_dist;  // every table entry's distance sqrt_hw(FP32 squared distance), same
                            // layout; table_pairs: float2 {distance, target value} per entry
  int32_t table_pairs;    // 1: the tables store (distance, target value) pairs (TableJob::tv_i)
  int32_t table_u16;      // 1: uint16 entries (every manifold below 65536 points), 0: int32
  double* partials;       // 6 doubles per query tile
  const double* obs;      // observed-moment tile records (TargetDesc::obs_tile)
  uint32_t* unit_done;    // per-unit tile counters (reset by the unit's last tile)
  uint32_t* item_counter; // dynamic scheduling counter (zeroed before each launch)
  double* rho;            // output (device), indexed by UnitDesc::out_idx
  int32_t* dbg_nbr;       // optional [sum N_m][E+1]
  float* dbg_xhat;        // optional [sum N_m]
  int32_t* err;
  unsigned long long* stats;  // optional search counters [kStatCount] (kStat*), nullptr: none
  int32_t persistent;     // 1: CTAs pull items from item_counter; 0: item = blockIdx.x
  int32_t merge_at[kMaxE + 1];  // per E: merge pending candidates once a lane holds this many
  int32_t variant[kMaxE + 1];   // per E: kernel variant (0 narrow, 1 wide); same results
};

// Search counters, accumulated by the kernels when KnnParams::stats is set (a
// separately compiled counting variant; the results are the same).
enum : int {
  kStatBruteTiles = 0,   // query tiles searched by brute force
  kStatBruteQueries,     // their valid queries
  kStatPairsBegun,       // query-library pairs whose distance was begun (lanes x points)
  kStatPairsFull,        // pairs whose distance was completed over all E coordinates
  kStatPairsPruned,      // pairs skipped by chunk pruning (lanes x chunk points)
  kStatCandidates,       // candidates appended to the pending buffers
  kStatMergeSlots,       // lockstep insertion slots: per warp merge, 32 x its largest pending count
  kStatTableQueries,     // valid queries answered from a distance indexing table
  kStatTableEntries,     // table entries loaded (per lane, eight per step)
  kStatTableFallbacks,   // queries that scanned their library instead
  kStatCount = 16
};

// Defaults before tuning: merge trigger (pending candidates per lane) and variant.
constexpr int kDefaultMergeAt = 4;
constexpr int kDefaultVariant = 1;

// Hardware square root and reciprocal (sqrt.approx.f32, rcp.approx.f32:
// within about one ulp, subnormal inputs included).
__device__ __forceinline__ float sqrt_hw(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_hw(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Simplex weight (paper Sect. 2.1) of a neighbour at distance d = sqrt_hw(d2)
// when the nearest is at distance d1 (> 0; inv_d1 = rcp_hw(d1)): u =
// exp(-d/d1), raised to the floor f.  d1 = 0 takes the limit: 1 for d = 0,
// else 0.  Shared by the fused kernels and the plain comparator so that all
// compute the same bits; FP32 with the hardware square root, reciprocal and
// exponential (relative error near 1e-7, far inside the 1e-5 the predictions
// are checked to).  The two cases separately, then together:
__device__ __forceinline__ float simplex_exp(float d, float inv_d1) {  // d1 > 0
  return __expf(-__fmul_rn(d, inv_d1));
}
__device__ __forceinline__ float simplex_limit(float d) {  // d1 = 0
  return (d == 0.f) ? 1.f : 0.f;
}
__device__ __forceinline__ float simplex_u_dist(float d, float d1, float inv_d1, float wfloor) {
  return fmaxf((d1 > 0.f) ? simplex_exp(d, inv_d1) : simplex_limit(d), wfloor);
}
__device__ __forceinline__ float simplex_u(float d2, float d1, float inv_d1, float wfloor) {
  return simplex_u_dist(sqrt_hw(d2), d1, inv_d1, wfloor);
}

// Error flag values written by kernels.
constexpr int32_t kErrBadUnit = 1;
constexpr int32_t kErrSampler = 2;

// Sampler (sampler.cu).
constexpr int kSamplerThreads = 256;
constexpr int kSamplerSmemKeys = 40960;   // keys kept in shared memory up to this N_m
cudaError_t sampler_prepare();
cudaError_t launch_sampler(const SamplerParams& p, int64_t first_unit, int64_t count,
                           int max_nm, cudaStream_t s);

// Query order (order.cu).
cudaError_t order_prepare();
cudaError_t launch_order(const float* series, const OrderJob* jobs, int64_t n_jobs, int max_nm,
                         int32_t* order, unsigned long long* scratch, cudaStream_t s);

// Distance indexing table (table.cu).
cudaError_t table_prepare();
// One launch builds the tables of jobs[0..n_jobs), all of embedding dimension E.
cudaError_t launch_table_build(const float* series, const TableJob* jobs, int64_t n_jobs, int E,
                               int max_nm, int max_R, const int32_t* order, void* table,
                               float* table_dist, int table_pairs, int table_u16, cudaStream_t s);

// Fused kernel (knn_fused.cu).
int knn_block_threads();
int knn_queries_per_thread();
cudaError_t knn_prepare();
cudaError_t knn_occupancy(int E, int* ctas_per_sm);
cudaError_t launch_knn(const KnnParams& p, int E, int grid, cudaStream_t s);
// Observed-moment records of every ObsJob (after the query order): one warp
// per tile, n_tiles tiles in all.
cudaError_t launch_obs(const float* series, const int32_t* order, const ObsJob* jobs,
                       int64_t n_jobs, int64_t n_tiles, double* obs, cudaStream_t s);
// Table path: same work items, neighbours read from the distance indexing table.
size_t knn_table_smem(int max_nm);
cudaError_t knn_table_prepare();
cudaError_t knn_table_occupancy(int max_nm, int* ctas_per_sm);
cudaError_t launch_knn_table(const KnnParams& p, int E, int max_nm, int grid, cudaStream_t s);

// Sets the thread-local message returned by ccm_last_error() (runtime.cu).
void set_last_error(const char* msg);

// Plain comparator (plain.cu): one realization per call.
// Convergence decision (one CTA per (pair, E, tau) row of the rho grid).
constexpr int kMaxConvGroups = 64;      // L values per row, at most
constexpr int kMaxConvValues = 24576;   // n_L * r per row, at most (shared memory)
struct ConvOrder {
  int32_t group[kMaxConvGroups];        // L-axis index of the g-th smallest L
};
struct ConvergenceRow {                 // same layout as ccm_convergence_t
  double rho_first, rho_last, jt, z;
  int32_t n_valid, converged;
};
cudaError_t convergence_prepare();
cudaError_t launch_convergence(const double* rho, int64_t n_rows, int32_t n_L, int32_t r,
                               const ConvOrder& ord, double z_crit, ConvergenceRow* out,
                               cudaStream_t s);

cudaError_t launch_plain_unit(const float* series, const UnitDesc* unit_dev, const UnitDesc& unit,
                              const TargetDesc* target_dev, const int32_t* lib,
                              float* xhat_scratch, double* rho_out, cudaStream_t s);

}  // namespace ccm
