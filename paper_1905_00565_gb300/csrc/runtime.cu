// Host runtime of the CCM library: the C ABI of include/ccm.h.
//
//  * context: device, device-memory budget, one-time kernel set-up, serving
//    thread;
//  * plan: validated copy of a problem, its realizations ("units") in output
//    order, the work list of (unit, query tile) items sorted by decreasing
//    cost, and one device arena for series, libraries, partial moments and rho;
//  * run: sampler launch + one persistent fused-kernel launch, captured once
//    into a CUDA graph and replayed;
//  * plain comparator: one launch sequence per realization;
//  * serving: queued jobs are admitted while their footprints fit the free
//    budget, admitted jobs are batched into shared launches on a pool of
//    streams, and results are copied back per job.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <sys/stat.h>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "ccm.h"
#include "ccm_internal.h"

using namespace ccm;

namespace {

thread_local std::string t_err;

ccm_status fail(ccm_status st, const std::string& msg) {
  t_err = msg;
  return st;
}

#define CCM_CUDA(call)                                                                   \
  do {                                                                                   \
    const cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                               \
      return fail(CCM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- problem ---
struct ProblemCopy {
  int32_t V = 0;
  int64_t n = 0;
  std::vector<int32_t> pairs, E, tau;
  std::vector<int64_t> L;
  int32_t r = 0;
  uint64_t seed = 0;
  uint32_t flags = 0;
  int32_t theiler = 0;
  float weight_floor = 0.f;

  int64_t n_units() const {
    return (int64_t)(pairs.size() / 2) * (int64_t)E.size() * (int64_t)tau.size() *
           (int64_t)L.size() * r;
  }
};

ccm_status copy_problem(const ccm_problem* p, ProblemCopy* pc) {
  if (!p) return fail(CCM_EINVAL, "problem is NULL");
  if (p->n_series < 2) return fail(CCM_EINVAL, "n_series must be >= 2");
  if (p->n < 3 || p->n > 0x7fffffff) return fail(CCM_EINVAL, "series length out of range");
  if (p->n_pairs < 1 || !p->pairs) return fail(CCM_EINVAL, "no pairs");
  if (p->n_E < 1 || !p->E || p->n_tau < 1 || !p->tau || p->n_L < 1 || !p->L)
    return fail(CCM_EINVAL, "empty E, tau or L grid");
  if (p->r < 1) return fail(CCM_EINVAL, "r must be >= 1");
  pc->V = p->n_series;
  pc->n = p->n;
  pc->pairs.assign(p->pairs, p->pairs + 2 * (size_t)p->n_pairs);
  pc->E.assign(p->E, p->E + p->n_E);
  pc->tau.assign(p->tau, p->tau + p->n_tau);
  pc->L.assign(p->L, p->L + p->n_L);
  pc->r = p->r;
  pc->seed = p->seed;
  pc->flags = p->flags;
  if (p->flags & ~(uint32_t)(CCM_INPUT_ON_DEVICE | CCM_OUTPUT_ON_DEVICE | CCM_NO_AUTOTUNE |
                             CCM_NO_TABLE | CCM_SEARCH_STATS))
    return fail(CCM_EINVAL, "unknown flag bits");
  pc->theiler = p->theiler;
  pc->weight_floor = p->weight_floor;
  if (p->theiler < 0) return fail(CCM_EINVAL, "theiler window must be >= 0");
  if (!std::isfinite(p->weight_floor) || p->weight_floor < 0.f)
    return fail(CCM_EINVAL, "weight_floor must be finite and >= 0");
  for (int32_t q = 0; q < p->n_pairs; ++q) {
    const int32_t j = pc->pairs[2 * q], i = pc->pairs[2 * q + 1];
    if (j < 0 || j >= pc->V || i < 0 || i >= pc->V || i == j)
      return fail(CCM_EINVAL, "pair " + std::to_string(q) + " is invalid (need 0<=i,j<V, i!=j)");
  }
  {
    // a realization completes after (query tiles) x (targets of its library
    // variable) reductions, counted in 32 bits
    std::map<int32_t, int64_t> targets_of;
    int64_t most = 0;
    for (int32_t q = 0; q < p->n_pairs; ++q) most = std::max(most, ++targets_of[pc->pairs[2 * q]]);
    if (most * ((pc->n + 255) / 256) > 0x7fffffff)
      return fail(CCM_EINVAL, "targets of one library variable x query tiles exceed 2^31 - 1");
  }
  for (int32_t E : pc->E)
    if (E < 1 || E > kMaxE) return fail(CCM_EINVAL, "E must be in 1..10");
  for (int32_t t : pc->tau)
    if (t < 1) return fail(CCM_EINVAL, "tau must be >= 1");
  for (int32_t E : pc->E)
    for (int32_t t : pc->tau) {
      const int64_t n_m = pc->n - (int64_t)(E - 1) * t;
      for (int64_t L : pc->L) {
        if (L < E + 2 || L > n_m)
          return fail(CCM_EINVAL, "L=" + std::to_string(L) + " outside [E+2, N_m] for E=" +
                                      std::to_string(E) + ", tau=" + std::to_string(t));
        if (L < (int64_t)E + 2 + 2 * (int64_t)pc->theiler)
          return fail(CCM_EINVAL, "L=" + std::to_string(L) + " < E+2+2W for E=" +
                                      std::to_string(E) + ", W=" + std::to_string(pc->theiler));
      }
    }
  if ((double)pc->n_units() > 2.0e9) return fail(CCM_EINVAL, "too many realizations");
  return CCM_OK;
}

bool all_finite(const float* x, size_t count) {
  for (size_t q = 0; q < count; ++q)
    if (!std::isfinite(x[q])) return false;
  return true;
}

// ------------------------------------------------------------- unit lists ---
struct UnitList {
  std::vector<UnitDesc> units;        // library realizations
  std::vector<TargetDesc> targets;    // their targets (one per output rho)
  std::vector<WorkItem> items;        // brute-force items, grouped by E (see sort_items)
  std::vector<double> item_cost;
  int64_t e_first[kMaxE + 1] = {};    // items of E: e_count[E] from index e_first[E]
  int64_t e_count[kMaxE + 1] = {};
  int64_t te_first[kMaxE + 1] = {};   // the same for the table items
  int64_t te_count[kMaxE + 1] = {};
  std::vector<OrderJob> orders;       // one per (job, library variable, E, tau)
  std::vector<ObsJob> obs_jobs;       // one per (job, library variable, target, E, tau)
  int64_t obs_total = 0;              // observed-moment tile records
  std::vector<TableJob> tables;       // distance indexing tables to build
  std::vector<WorkItem> items_table;  // work items of units that read a table
  std::vector<double> item_cost_table;
  int64_t lib_total = 0, part_total = 0, order_total = 0, table_total = 0;
  int64_t order_scratch_total = 0;    // 64-bit keys for sorting manifolds above kOrderMaxSort
  // Table jobs are sorted by (sort size, E) (sort_items) and built one launch
  // per sort size (the power of two at or above R) and E: a launch's shared
  // memory per warp follows its own largest row, so short rows run more warps
  // per SM, and its registers follow its E.
  static int table_rcap(int R) {
    int rc = 32;
    while (rc < R) rc <<= 1;
    return rc;
  }
  int table_groups() const {
    int g = 0;
    for (size_t q = 0; q < tables.size(); ++q)
      if (q == 0 || table_rcap(tables[q].R) != table_rcap(tables[q - 1].R) ||
          tables[q].E != tables[q - 1].E)
        ++g;
    return g;
  }
  double brute_flops = 0.0;           // 3E per pair of the units searched by brute force
  double brute_pairs = 0.0;           // query-library pairs of those units
  int64_t search_queries = 0;         // N_m summed over the units
  int64_t table_queries = 0;          // N_m summed over the units that read a table
  bool table_tv = false;              // some table stores its target's values (TableJob::tv_i)
  int table_u16() const { return max_nm < 65536 ? 1 : 0; }
  size_t table_elem() const { return table_u16() ? 2 : 4; }
  int64_t n_rho = 0, q_total = 0, nbr_total = 0, lib_dbg_total = 0;  // per output realization
  int emin = kMaxE + 1, emax = 0, max_nm = 0;
  double pairs = 0.0, flops = 0.0;    // neighbour-search work actually done
};

// Table tunables: the crossover constant c, the floor and the largest
// manifold-to-library ratio of table_min_L, and a factor s on the row length
// (see below).  The environment variables CCM_TABLE_CROSSOVER, CCM_TABLE_FLOOR,
// CCM_TABLE_MAX_RATIO and CCM_TABLE_SAFETY replace the defaults (read at each
// ccm_plan; tuning and measurement only).
struct TableTuning {
  double crossover, floor, max_ratio, safety;
};
TableTuning read_table_tuning() {
  TableTuning r{20.0, 256.0, 40.0, 1.0};
  if (const char* e = getenv("CCM_TABLE_CROSSOVER")) r.crossover = std::max(0.0, atof(e));
  if (const char* e = getenv("CCM_TABLE_FLOOR")) r.floor = std::max(16.0, atof(e));
  if (const char* e = getenv("CCM_TABLE_MAX_RATIO")) r.max_ratio = std::max(1.0, atof(e));
  if (const char* e = getenv("CCM_TABLE_SAFETY")) r.safety = std::max(0.01, atof(e));
  return r;
}

// Smallest L whose realizations read a distance indexing table.  A table
// walk visits about (E+1)*N_m/L row entries per query; brute force (with chunk
// pruning) costs about L distance evaluations of E coordinates per query, far
// fewer at small E, where pruning skips most chunks.  Measured on GB300: on
// the N_m = 10^4 sweep (the table build included) c = 20 and a floor of 256
// are fastest, L ~ sqrt(c*N_m/(E+1)) being where a grouped table walk
// overtakes the selection-bound brute force of small libraries; on the
// N = 10^5 series (E = 3..6) brute force at L = 1000 beats walks of
// (E+1)*100 entries, so libraries below N_m/max_ratio (40) points stay with
// brute force.  The last term keeps the row length (table_row_length) within
// kTableMaxR.
double table_min_L(int32_t E, int64_t n_m, const TableTuning& t) {
  return std::max({t.floor, std::ceil(std::sqrt(t.crossover * (double)n_m / (double)(E + 1))),
                   std::ceil((double)n_m / t.max_ratio),
                   std::ceil(t.safety * 2.8 * (E + 2) * (double)n_m / (double)kTableMaxR)});
}

// Row length R of a table whose smallest L is lmin.  A query of a realization
// with L = lmin finds a Poisson(lambda = R*lmin/N_m) number of its library's
// points among its R entries (the library is a uniform sample); with fewer
// than E+1 it scans its whole library instead, about lmin distance
// evaluations.  lambda is the smallest multiple of 1/4 for which that happens
// with probability at most 1/(10*lmin), so the misses cost at most about 0.1
// distance evaluations a query (times the safety factor s on lambda); 2W more
// entries cover the points the exclusion window removes.
int64_t table_row_length(int32_t E, int64_t n_m, int64_t lmin, int32_t theiler, double safety) {
  const double eps = 1.0 / (10.0 * (double)lmin);
  double lambda = (double)(E + 1);
  for (;; lambda += 0.25) {
    double term = std::exp(-lambda), tail = term;  // P(X <= E), X ~ Poisson(lambda)
    for (int i = 1; i <= E; ++i) {
      term *= lambda / i;
      tail += term;
    }
    if (tail <= eps) break;
  }
  return (int64_t)std::ceil(safety * lambda * (double)n_m / (double)lmin) + 2 * (int64_t)theiler;
}

// Append the units of one problem.  Offsets: series block, first rho index.
// Pairs that share a library variable j share one library and one neighbour
// search per (E, tau, L, k); each pair becomes a target of that unit.
void append_units(const ProblemCopy& pc, int64_t series_off, int64_t out_base, UnitList* ul,
                  double table_cap_bytes) {
  const int tileq = knn_block_threads() * knn_queries_per_thread();
  const int64_t nP = (int64_t)pc.pairs.size() / 2;
  const int64_t nE = (int64_t)pc.E.size(), nT = (int64_t)pc.tau.size(), nL = (int64_t)pc.L.size();
  const int64_t per_pair = nE * nT * nL * pc.r;
  // debug offsets of every output realization, in rho order
  std::vector<int64_t> q_off((size_t)(nP * per_pair)), nbr_off(q_off.size()), lib_off(q_off.size());
  {
    int64_t o = 0;
    for (int64_t p = 0; p < nP; ++p)
      for (int32_t E : pc.E)
        for (int32_t tau : pc.tau)
          for (int64_t L : pc.L)
            for (int32_t k = 0; k < pc.r; ++k, ++o) {
              const int64_t n_m = pc.n - (int64_t)(E - 1) * tau;
              q_off[(size_t)o] = ul->q_total;
              nbr_off[(size_t)o] = ul->nbr_total;
              lib_off[(size_t)o] = ul->lib_dbg_total;
              ul->q_total += n_m;
              ul->nbr_total += n_m * (E + 1);
              ul->lib_dbg_total += L;
            }
    ul->n_rho += o;
  }
  // library variables in order of first appearance, with their pairs
  std::vector<int32_t> lib_vars;
  std::map<int32_t, std::vector<int64_t>> pairs_of;
  for (int64_t p = 0; p < nP; ++p) {
    const int32_t j = pc.pairs[2 * p];
    if (!pairs_of.count(j)) lib_vars.push_back(j);
    pairs_of[j].push_back(p);
  }
  std::map<std::tuple<int32_t, int32_t, int32_t>, int64_t> combo;  // (j, E, tau) -> order_off
  for (int32_t j : lib_vars)
    for (int32_t E : pc.E)
      for (int32_t tau : pc.tau) {
        OrderJob oj;
        std::memset(&oj, 0, sizeof(oj));
        oj.series_off = series_off;
        oj.n = pc.n;
        oj.order_off = ul->order_total;
        oj.scratch_off = -1;
        oj.j = j;
        oj.E = E;
        oj.tau = tau;
        oj.n_m = (int32_t)(pc.n - (int64_t)(E - 1) * tau);
        combo[std::make_tuple(j, E, tau)] = oj.order_off;
        ul->order_total += oj.n_m;
        if (oj.n_m > kOrderMaxSort) {
          oj.scratch_off = ul->order_scratch_total;
          ul->order_scratch_total += 2 * (int64_t)oj.n_m;
        }
        ul->orders.push_back(oj);
      }
  // Observed-moment records per (j, i, E, tau), shared by every L and k.
  std::map<std::tuple<int32_t, int32_t, int32_t, int32_t>, int64_t> obs_of;
  for (int32_t j : lib_vars)
    for (int64_t p : pairs_of[j])
      for (int32_t E : pc.E)
        for (int32_t tau : pc.tau) {
          const int32_t i = pc.pairs[2 * p + 1];
          const auto key = std::make_tuple(j, i, E, tau);
          if (obs_of.count(key)) continue;
          ObsJob ob;
          std::memset(&ob, 0, sizeof(ob));
          ob.series_off = series_off;
          ob.n = pc.n;
          ob.order_off = combo[std::make_tuple(j, E, tau)];
          ob.obs_tile = ul->obs_total;
          ob.i = i;
          ob.E = E;
          ob.tau = tau;
          ob.n_m = (int32_t)(pc.n - (int64_t)(E - 1) * tau);
          ob.n_tiles = (ob.n_m + tileq - 1) / tileq;
          obs_of[key] = ob.obs_tile;
          ul->obs_total += ob.n_tiles;
          ul->obs_jobs.push_back(ob);
        }
  // Distance indexing tables (unless CCM_NO_TABLE): per (j, E, tau),
  // realizations with L >= table_min_L read their neighbours from a table of
  // the R nearest points of every query (R from table_row_length at the
  // smallest such L).  A table is built only when the
  // realizations that use it would otherwise scan at least 8*N_m library
  // points in total (its build costs about N_m^2 distance evaluations), and
  // while the plan's tables stay within table_cap_bytes; the realizations of
  // a (j, E, tau) without a table use brute force.
  std::map<std::tuple<int32_t, int32_t, int32_t>, std::pair<int64_t, int32_t>> table_of;
  // The safety factor trades table memory and build time against how often a
  // query falls back to scanning its library.
  const TableTuning tt = read_table_tuning();
  const double safety = tt.safety;
  double table_bytes = 0.0;
  if (!(pc.flags & CCM_NO_TABLE)) {
    for (int32_t j : lib_vars)
      for (int32_t E : pc.E)
        for (int32_t tau : pc.tau) {
          const int64_t n_m = pc.n - (int64_t)(E - 1) * tau;
          if (n_m > kTableMaxNm) continue;
          const double ls = table_min_L(E, n_m, tt);
          int64_t lmin = -1;
          double lsum = 0.0;
          for (int64_t L : pc.L)
            if ((double)L >= ls) {
              lmin = (lmin < 0) ? L : std::min(lmin, L);
              lsum += (double)L * pc.r;
            }
          if (lmin < 0 || lsum < 8.0 * (double)n_m) continue;
          int64_t R = table_row_length(E, n_m, lmin, pc.theiler, safety);
          // whole groups of four ranks (the table's layout), from the n_m - 1
          // points other than the query
          R = std::min<int64_t>(std::min<int64_t>((R + 31) / 32 * 32, kTableMaxR),
                                (n_m - 1) / 4 * 4);
          // indices (2 or 4 bytes), distances, and (a variable with one target,
          // a manifold below 65536 points) the target's values: the scan then
          // reads them beside the distances instead of gathering them through
          // the indices (on longer manifolds the extra array's cold lines cost
          // more than the gather: 120 -> 129 ms on the N = 10^5 series)
          const bool tv = pairs_of[j].size() == 1 && n_m < 65536;
          const double bytes =
              (double)n_m * (double)R * ((n_m < 65536 ? 2.0 : 4.0) + 4.0 + (tv ? 4.0 : 0.0));
          if (table_bytes + bytes > table_cap_bytes) continue;
          table_bytes += bytes;
          TableJob tj;
          std::memset(&tj, 0, sizeof(tj));
          tj.series_off = series_off;
          tj.n = pc.n;
          tj.order_off = combo[std::make_tuple(j, E, tau)];
          tj.table_off = ul->table_total;
          tj.j = j;
          tj.E = E;
          tj.tau = tau;
          tj.n_m = (int32_t)n_m;
          tj.R = (int32_t)R;
          tj.tv_i = tv ? pc.pairs[2 * pairs_of[j][0] + 1] : -1;
          if (tv) ul->table_tv = true;
          table_of[std::make_tuple(j, E, tau)] = std::make_pair(tj.table_off, tj.R);
          ul->table_total += n_m * R;
          ul->tables.push_back(tj);
        }
  }
  for (int32_t j : lib_vars) {
    const std::vector<int64_t>& tp = pairs_of[j];
    for (int64_t e = 0; e < nE; ++e)
      for (int64_t t = 0; t < nT; ++t)
        for (int64_t l = 0; l < nL; ++l)
          for (int32_t k = 0; k < pc.r; ++k) {
            const int32_t E = pc.E[(size_t)e], tau = pc.tau[(size_t)t];
            const int64_t L = pc.L[(size_t)l];
            UnitDesc u;
            std::memset(&u, 0, sizeof(u));
            u.series_off = series_off;
            u.n = pc.n;
            u.j = j;
            u.E = E;
            u.tau = tau;
            u.L = (int32_t)L;
            u.k = k;
            u.seed = pc.seed;
            u.n_m = (int32_t)(pc.n - (int64_t)(E - 1) * tau);
            u.n_tiles = (u.n_m + tileq - 1) / tileq;
            u.n_targets = (int32_t)tp.size();
            u.theiler = pc.theiler;
            u.wfloor = pc.weight_floor;
            u.lib_off = ul->lib_total;
            u.part_off = ul->part_total;
            u.order_off = combo[std::make_tuple(j, E, tau)];
            u.tgt_off = (int64_t)ul->targets.size();
            for (int64_t p : tp) {
              const int64_t o = (((p * nE + e) * nT + t) * nL + l) * pc.r + k;  // rho order
              TargetDesc tg;
              std::memset(&tg, 0, sizeof(tg));
              tg.out_idx = out_base + o;
              tg.q_off = q_off[(size_t)o];
              tg.nbr_off = nbr_off[(size_t)o];
              tg.lib_dbg_off = lib_off[(size_t)o];
              tg.i = pc.pairs[2 * p + 1];
              tg.obs_tile = obs_of[std::make_tuple(j, tg.i, E, tau)];
              ul->targets.push_back(tg);
            }
            const auto tab = table_of.find(std::make_tuple(j, E, tau));
            if (tab != table_of.end() && (double)L >= table_min_L(E, u.n_m, tt)) {
              u.table_off = tab->second.first;
              u.table_R = tab->second.second;
              u.table_tv = (tp.size() == 1 && u.n_m < 65536) ? 1 : 0;  // as the table's job
            }
            const int32_t uidx = (int32_t)ul->units.size();
            // Table realizations of one cell with a single target and a byte
            // membership map are grouped kTableGroup at a time (consecutive k):
            // the item of the group's first realization covers all of them.
            const bool groupable = u.table_R > 0 && u.n_targets == 1 && u.n_m <= kTableGroupMaxNm;
            const int32_t count =
                groupable ? std::min<int32_t>(kTableGroup, pc.r - (k / kTableGroup) * kTableGroup) : 1;
            const bool owns_items = !groupable || k % kTableGroup == 0;
            for (int32_t q = 0; q < u.n_tiles && owns_items; ++q) {
              const int64_t nq = std::min<int64_t>(tileq, u.n_m - (int64_t)q * tileq);
              if (u.table_R > 0) {
                // one item per kTableChunk tiles: one membership map, then per
                // tile one walk of each row (longer for a group: it ends when
                // every realization has its E+1) and one epilogue per
                // realization and target
                if (q % kTableChunk == 0) {
                  ul->items_table.push_back(WorkItem{uidx, q, count});
                  ul->item_cost_table.push_back((double)L * count);
                }
                ul->item_cost_table.back() +=
                    (double)nq * 12.0 * (E + 2) * (double)u.n_m / (double)L * (1.0 + 0.1 * count) +
                    (double)u.n_targets * nq * 64.0 * count;
              } else {
                // one item per kBruteChunk tiles: one library staging (when it
                // fits a shared-memory tile), then per tile the search and the
                // per-target epilogue
                if (q % kBruteChunk == 0) {
                  ul->items.push_back(WorkItem{uidx, q, 1});
                  ul->item_cost.push_back(64.0 * E * (double)L);
                }
                ul->item_cost.back() += (double)L * (double)nq * (2.0 * E + 1.0) +
                                        (double)u.n_targets * nq * 64.0;
              }
            }
            if (u.table_R == 0) {
              ul->brute_flops += 3.0 * E * (double)u.n_m * (double)L;
              ul->brute_pairs += (double)u.n_m * (double)L;
            } else {
              ul->table_queries += u.n_m;
            }
            ul->search_queries += u.n_m;
            ul->lib_total += L;
            ul->part_total += (int64_t)u.n_tiles * u.n_targets;
            ul->emin = std::min(ul->emin, E);
            ul->emax = std::max(ul->emax, E);
            ul->max_nm = std::max(ul->max_nm, u.n_m);
            ul->pairs += (double)u.n_m * (double)L;
            ul->flops += 3.0 * E * (double)u.n_m * (double)L;
            ul->units.push_back(u);
          }
  }
}

void sort_items(UnitList* ul) {
  std::stable_sort(ul->tables.begin(), ul->tables.end(), [](const TableJob& a, const TableJob& b) {
    const int ra = UnitList::table_rcap(a.R), rb = UnitList::table_rcap(b.R);
    if (ra != rb) return ra < rb;
    if (a.E != b.E) return a.E < b.E;
    return a.R < b.R;
  });
  // Brute-force items: grouped by E (one single-E kernel launch per group,
  // in the stream's order), larger items first within a group.
  {
    std::vector<int64_t> order(ul->items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int64_t)q;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      const int32_t ea = ul->units[(size_t)ul->items[(size_t)a].unit].E;
      const int32_t eb = ul->units[(size_t)ul->items[(size_t)b].unit].E;
      if (ea != eb) return ea > eb;
      return ul->item_cost[(size_t)a] > ul->item_cost[(size_t)b];
    });
    std::vector<WorkItem> sorted(order.size());
    std::vector<double> cost(order.size());
    for (size_t q = 0; q < order.size(); ++q) {
      sorted[q] = ul->items[(size_t)order[q]];
      cost[q] = ul->item_cost[(size_t)order[q]];
    }
    ul->items.swap(sorted);
    ul->item_cost.swap(cost);
    for (int E = 0; E <= kMaxE; ++E) ul->e_first[E] = ul->e_count[E] = 0;
    for (const WorkItem& w : ul->items) ++ul->e_count[ul->units[(size_t)w.unit].E];
    int64_t at = 0;  // groups are stored from E = 10 down to E = 1
    for (int E = kMaxE; E >= 1; --E) {
      ul->e_first[E] = at;
      at += ul->e_count[E];
    }
  }
  // Table items: grouped by E (one launch per E), then by table (a table of
  // 5-30 MB stays in L2 while its realizations run), larger items first.
  std::vector<int64_t> order(ul->items_table.size());
  for (size_t q = 0; q < order.size(); ++q) order[q] = (int64_t)q;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const UnitDesc& ua = ul->units[(size_t)ul->items_table[(size_t)a].unit];
    const UnitDesc& ub = ul->units[(size_t)ul->items_table[(size_t)b].unit];
    if (ua.E != ub.E) return ua.E > ub.E;
    if (ua.table_off != ub.table_off) return ua.table_off < ub.table_off;
    return ul->item_cost_table[(size_t)a] > ul->item_cost_table[(size_t)b];
  });
  std::vector<WorkItem> sorted(order.size());
  for (size_t q = 0; q < order.size(); ++q) sorted[q] = ul->items_table[(size_t)order[q]];
  ul->items_table.swap(sorted);
  for (int E = 0; E <= kMaxE; ++E) ul->te_first[E] = ul->te_count[E] = 0;
  for (const WorkItem& w : ul->items_table) ++ul->te_count[ul->units[(size_t)w.unit].E];
  int64_t at = 0;
  for (int E = kMaxE; E >= 1; --E) {
    ul->te_first[E] = at;
    at += ul->te_count[E];
  }
}

// Device arena layout for a unit list.
struct Arena {
  size_t series = 0, units = 0, items = 0, lib = 0, part = 0, done = 0, rho = 0, err = 0,
         counter = 0, scratch = 0, order = 0, orders = 0, targets = 0, table = 0, tables = 0,
         items_table = 0, order_scratch = 0, obs = 0, obs_jobs = 0, table_dist = 0, stats = 0,
         total = 0;
};

Arena layout(int64_t series_elems, const UnitList& ul, int64_t n_rho, int64_t scratch_floats) {
  Arena a;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  a.series = take(sizeof(float) * (size_t)series_elems);
  a.units = take(sizeof(UnitDesc) * ul.units.size());
  a.items = take(sizeof(WorkItem) * ul.items.size());
  a.lib = take(sizeof(int32_t) * (size_t)ul.lib_total);
  a.part = take(6 * sizeof(double) * (size_t)ul.part_total);
  a.done = take(sizeof(uint32_t) * ul.units.size());
  a.rho = take(sizeof(double) * (size_t)n_rho);
  a.err = take(sizeof(int32_t));
  a.counter = take(2 * (kMaxE + 1) * sizeof(uint32_t));  // [E] brute force, [kMaxE+1+E] table
  a.scratch = take(sizeof(float) * (size_t)scratch_floats);
  a.order = take(sizeof(int32_t) * (size_t)ul.order_total);
  a.order_scratch = take(sizeof(unsigned long long) * (size_t)ul.order_scratch_total);
  a.orders = take(sizeof(OrderJob) * ul.orders.size());
  a.targets = take(sizeof(TargetDesc) * ul.targets.size());
  a.table = take(ul.table_elem() * (size_t)ul.table_total);
  a.table_dist = take((ul.table_tv ? sizeof(float2) : sizeof(float)) * (size_t)ul.table_total);
  a.tables = take(sizeof(TableJob) * ul.tables.size());
  a.items_table = take(sizeof(WorkItem) * ul.items_table.size());
  a.obs = take(sizeof(double) * kObsStride * (size_t)ul.obs_total);
  a.obs_jobs = take(sizeof(ObsJob) * ul.obs_jobs.size());
  a.stats = take(sizeof(unsigned long long) * kStatCount);
  a.total = o;
  return a;
}

}  // namespace

namespace ccm {
void set_last_error(const char* msg) { t_err = msg; }
}  // namespace ccm

// Per-E kernel parameters chosen by the autotuner (results do not depend on them).
struct Tuning {
  int32_t variant[kMaxE + 1];
  int32_t merge_at[kMaxE + 1];
  bool known[kMaxE + 1];  // chosen by measurement (here or from the cache)
};

Tuning default_tuning() {
  Tuning t;
  for (int e = 0; e <= kMaxE; ++e) {
    t.variant[e] = kDefaultVariant;
    t.merge_at[e] = kDefaultMergeAt;
    t.known[e] = false;
  }
  return t;
}

// ================================================================ context ===
struct Job;
struct Batch;

struct ccm_context {
  int device = 0;
  std::string device_name;
  Tuning tuning = default_tuning();  // per-E choices known to this context (cache + runs)
  size_t budget = 0;
  size_t used = 0;
  int sm_count = 0;
  std::mutex mu;  // budget, job table, queue, batches
  std::condition_variable cv;
  // serving state
  std::thread server;
  bool server_started = false;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::deque<std::shared_ptr<Job>> queue;
  std::list<std::shared_ptr<Batch>> inflight;
  std::vector<cudaStream_t> streams;       // low priority: batches of large jobs
  std::vector<cudaStream_t> fast_streams;  // high priority: batches of small jobs
  size_t next_stream = 0, next_fast = 0;
  int max_inflight = 8;
  double batch_pairs = 5.0e10;             // query-library pairs per batch of small jobs
  // Test hook (CCM_FAULT_INJECT_BATCH, read at creation): the launch of batch
  // number inject_batch (0-based, in launch order) fails on the host as if a
  // CUDA call had returned an error; -1: off.  No device work is faulted.
  int64_t inject_batch = -1;
  int64_t batches_launched = 0;
  // Pinned staging buffers are pooled: cudaMallocHost/cudaFreeHost may
  // synchronise the device, which would stall polls and new batches behind a
  // running large job.  Size classes are powers of two.
  std::mutex pool_mu;
  std::multimap<size_t, void*> pool_free;
  std::vector<void*> pool_all;
};

namespace {
// Device memory the distance indexing tables of one plan (or served batch)
// may take: a quarter of the context's budget.
double table_cap(const ccm_context* ctx) { return 0.25 * (double)ctx->budget; }
}  // namespace

namespace {

size_t pool_class(size_t bytes) {
  size_t c = 256;
  while (c < bytes) c <<= 1;
  return c;
}

void* pinned_get(ccm_context* ctx, size_t bytes) {
  const size_t c = pool_class(bytes);
  std::lock_guard<std::mutex> g(ctx->pool_mu);
  auto it = ctx->pool_free.find(c);
  if (it != ctx->pool_free.end()) {
    void* ptr = it->second;
    ctx->pool_free.erase(it);
    return ptr;
  }
  void* ptr = nullptr;
  if (cudaMallocHost(&ptr, c) != cudaSuccess) return nullptr;
  ctx->pool_all.push_back(ptr);
  return ptr;
}

void pinned_put(ccm_context* ctx, void* ptr, size_t bytes) {
  if (!ptr) return;
  std::lock_guard<std::mutex> g(ctx->pool_mu);
  ctx->pool_free.emplace(pool_class(bytes), ptr);
}

ccm_status reserve(ccm_context* ctx, size_t bytes) {
  std::lock_guard<std::mutex> g(ctx->mu);
  if (bytes > ctx->budget)
    return fail(CCM_ETOOLARGE, "footprint " + std::to_string(bytes) + " B exceeds budget " +
                                   std::to_string(ctx->budget) + " B");
  if (ctx->used + bytes > ctx->budget)
    return fail(CCM_ENOMEM, "budget in use: " + std::to_string(ctx->used) + " of " +
                                std::to_string(ctx->budget) + " B");
  ctx->used += bytes;
  return CCM_OK;
}

void release(ccm_context* ctx, size_t bytes) {
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->used -= std::min(ctx->used, bytes);
}

}  // namespace

// =================================================================== plan ===
struct ccm_plan_s {
  ccm_context* ctx = nullptr;
  ProblemCopy pc;
  UnitList ul;
  Arena ar;
  char* d_arena = nullptr;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // stage boundaries
  int grid = 0, grid_table = 0;
  Tuning tuning = default_tuning();
  bool tuned = false;
  std::mutex run_mu;
  ccm_plan_info info{};
};

namespace {

SamplerParams sampler_params(char* base, const Arena& ar) {
  SamplerParams sp{};
  sp.units = reinterpret_cast<const UnitDesc*>(base + ar.units);
  sp.targets = reinterpret_cast<const TargetDesc*>(base + ar.targets);
  sp.order = reinterpret_cast<const int32_t*>(base + ar.order);
  sp.lib = reinterpret_cast<int32_t*>(base + ar.lib);
  sp.err = reinterpret_cast<int32_t*>(base + ar.err);
  return sp;
}

KnnParams knn_params(char* base, const Arena& ar, const UnitList& ul, int persistent,
                     const Tuning& tn) {
  KnnParams kp{};
  kp.series = reinterpret_cast<const float*>(base + ar.series);
  kp.units = reinterpret_cast<const UnitDesc*>(base + ar.units);
  kp.targets = reinterpret_cast<const TargetDesc*>(base + ar.targets);
  kp.items = reinterpret_cast<const WorkItem*>(base + ar.items);
  kp.n_items = (int64_t)ul.items.size();
  kp.lib = reinterpret_cast<const int32_t*>(base + ar.lib);
  kp.order = reinterpret_cast<const int32_t*>(base + ar.order);
  kp.table = base + ar.table;
  kp.table_dist = reinterpret_cast<const float*>(base + ar.table_dist);
  kp.table_pairs = ul.table_tv ? 1 : 0;
  kp.table_u16 = ul.table_u16();
  kp.partials = reinterpret_cast<double*>(base + ar.part);
  kp.obs = reinterpret_cast<const double*>(base + ar.obs);
  kp.unit_done = reinterpret_cast<uint32_t*>(base + ar.done);
  kp.item_counter = reinterpret_cast<uint32_t*>(base + ar.counter);
  kp.rho = reinterpret_cast<double*>(base + ar.rho);
  kp.err = reinterpret_cast<int32_t*>(base + ar.err);
  kp.persistent = persistent;
  for (int e = 0; e <= kMaxE; ++e) {
    kp.merge_at[e] = tn.merge_at[e];
    kp.variant[e] = tn.variant[e];
  }
  return kp;
}

cudaError_t enqueue_obs(char* base, const Arena& ar, const UnitList& ul, cudaStream_t s) {
  return launch_obs(reinterpret_cast<const float*>(base + ar.series),
                    reinterpret_cast<const int32_t*>(base + ar.order),
                    reinterpret_cast<const ObsJob*>(base + ar.obs_jobs),
                    (int64_t)ul.obs_jobs.size(), ul.obs_total,
                    reinterpret_cast<double*>(base + ar.obs), s);
}

// Enqueue sampler + fused kernel for a whole unit list on stream s.
// Stage events (optional): ev[0] start, ev[1] after order, observed moments and table build,
// ev[2] after the sampler, ev[3] after the brute-force launch, ev[4] after the
// table-scan launch.
ccm_status enqueue_sweep(char* base, const Arena& ar, const UnitList& ul, const Tuning& tn,
                         int grid, int grid_table, int persistent, int32_t* dbg_lib,
                         int32_t* dbg_nbr, float* dbg_xhat, cudaStream_t s,
                         cudaEvent_t* ev = nullptr, bool capturing = false,
                         bool stats = false) {
  // Inside stream capture an event record becomes a graph node only with the
  // external flag; outside capture the plain record is the valid form.
  auto record = [&](cudaEvent_t e) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                     : cudaEventRecord(e, s);
  };
  CCM_CUDA(cudaMemsetAsync(base + ar.err, 0, sizeof(int32_t), s));
  CCM_CUDA(cudaMemsetAsync(base + ar.counter, 0, 2 * (kMaxE + 1) * sizeof(uint32_t), s));
  CCM_CUDA(cudaMemsetAsync(base + ar.done, 0, sizeof(uint32_t) * ul.units.size(), s));
  if (stats) CCM_CUDA(cudaMemsetAsync(base + ar.stats, 0, sizeof(unsigned long long) * kStatCount, s));
  if (ev) CCM_CUDA(record(ev[0]));
  CCM_CUDA(launch_order(reinterpret_cast<const float*>(base + ar.series),
                        reinterpret_cast<const OrderJob*>(base + ar.orders),
                        (int64_t)ul.orders.size(), ul.max_nm,
                        reinterpret_cast<int32_t*>(base + ar.order),
                        reinterpret_cast<unsigned long long*>(base + ar.order_scratch), s));
  CCM_CUDA(enqueue_obs(base, ar, ul, s));
  for (size_t g0 = 0; g0 < ul.tables.size();) {  // one launch per (sort size, E)
    const int rc = UnitList::table_rcap(ul.tables[g0].R), te = ul.tables[g0].E;
    size_t g1 = g0;
    int nm = 0, rmax = 0;
    for (; g1 < ul.tables.size() && UnitList::table_rcap(ul.tables[g1].R) == rc &&
           ul.tables[g1].E == te;
         ++g1) {
      nm = std::max(nm, ul.tables[g1].n_m);
      rmax = std::max(rmax, ul.tables[g1].R);
    }
    CCM_CUDA(launch_table_build(reinterpret_cast<const float*>(base + ar.series),
                                reinterpret_cast<const TableJob*>(base + ar.tables) + g0,
                                (int64_t)(g1 - g0), te, nm, rmax,
                                reinterpret_cast<const int32_t*>(base + ar.order),
                                base + ar.table, reinterpret_cast<float*>(base + ar.table_dist),
                                ul.table_tv ? 1 : 0,
                                ul.table_u16(), s));
    g0 = g1;
  }
  if (ev) CCM_CUDA(record(ev[1]));
  SamplerParams sp = sampler_params(base, ar);
  sp.dbg_lib = dbg_lib;
  CCM_CUDA(launch_sampler(sp, 0, (int64_t)ul.units.size(), ul.max_nm, s));
  if (ev) CCM_CUDA(record(ev[2]));
  KnnParams kp = knn_params(base, ar, ul, persistent, tn);
  kp.dbg_nbr = dbg_nbr;
  kp.dbg_xhat = dbg_xhat;
  if (stats) kp.stats = reinterpret_cast<unsigned long long*>(base + ar.stats);
  // One launch per E (a kernel specialised for one E keeps its registers for
  // that E); each drains its own queue, larger items first, so the launches
  // follow each other with short tails.
  for (int E = kMaxE; E >= 1; --E) {
    if (ul.e_count[E] == 0) continue;
    KnnParams ke = kp;
    ke.items = kp.items + ul.e_first[E];
    ke.n_items = ul.e_count[E];
    ke.item_counter = reinterpret_cast<uint32_t*>(base + ar.counter) + E;
    const int g = persistent ? grid : (int)std::min<int64_t>(ul.e_count[E], 0x7fffffff);
    CCM_CUDA(launch_knn(ke, E, g, s));
  }
  if (ev) CCM_CUDA(record(ev[3]));
  for (int E = kMaxE; E >= 1; --E) {
    if (ul.te_count[E] == 0) continue;
    KnnParams kt = kp;
    kt.items = reinterpret_cast<const WorkItem*>(base + ar.items_table) + ul.te_first[E];
    kt.n_items = ul.te_count[E];
    kt.item_counter = reinterpret_cast<uint32_t*>(base + ar.counter) + (kMaxE + 1) + E;
    const int g = persistent ? grid_table : (int)std::min<int64_t>(ul.te_count[E], 0x7fffffff);
    CCM_CUDA(launch_knn_table(kt, E, ul.max_nm, g, s));
  }
  if (ev) CCM_CUDA(record(ev[4]));
  return CCM_OK;
}

ccm_status check_err_flag(char* base, const Arena& ar, cudaStream_t s) {
  int32_t err = 0;
  CCM_CUDA(cudaMemcpyAsync(&err, base + ar.err, sizeof(err), cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  if (err != 0) return fail(CCM_ECUDA, "kernel reported error flag " + std::to_string(err));
  return CCM_OK;
}

int persistent_grid(ccm_context* ctx, int emin, int emax) {
  int per_sm = 1 << 30;  // the smallest occupancy of the plan's kernels
  for (int E = std::max(emin, 1); E <= std::min(emax, kMaxE); ++E) {
    int c = 1;
    if (knn_occupancy(E, &c) != cudaSuccess || c < 1) c = 1;
    per_sm = std::min(per_sm, c);
  }
  if (per_sm == (1 << 30)) per_sm = 1;
  return ctx->sm_count * per_sm;
}

}  // namespace

// ============================================================== autotuner ===
namespace {

// Per E the tuner times the kernel variants (narrow / wide) and merge triggers
// on a stratified sample of the plan's own work items and keeps the fastest.
// Every candidate computes the same result; only the time differs.  Choices
// are cached per (device name, E) in a tab-separated file: $CCM_AUTOTUNE_CACHE,
// else ~/.cache/ccm_gb300/autotune.tsv.
std::string cache_path() {
  if (const char* p = getenv("CCM_AUTOTUNE_CACHE")) return p;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/ccm_gb300/autotune_v2.tsv";
}

void load_cache(ccm_context* ctx) {
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    char name[256];
    int E = 0, v = 0, ma = 0;
    if (sscanf(line, "%255[^\t]\t%d\t%d\t%d", name, &E, &v, &ma) == 4 &&
        ctx->device_name == name && E >= 1 && E <= kMaxE && v >= 0 && v <= 1 && ma >= 1 &&
        ma <= 16) {
      ctx->tuning.variant[E] = v;
      ctx->tuning.merge_at[E] = ma;
      ctx->tuning.known[E] = true;
    }
  }
  fclose(f);
}

void save_cache(const ccm_context* ctx, int E, int v, int ma) {
  const std::string path = cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {  // mkdir -p of the parent, best effort
    std::string dir = path.substr(0, slash);
    for (size_t q = 1; q <= dir.size(); ++q)
      if (q == dir.size() || dir[q] == '/') {
        const std::string d = dir.substr(0, q);
        (void)mkdir(d.c_str(), 0755);
      }
  }
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s\t%d\t%d\t%d\n", ctx->device_name.c_str(), E, v, ma);
  fclose(f);
}

constexpr double kTunePairs = 2.0e11;   // plans smaller than this use known or default choices

ccm_status autotune(ccm_plan_s* pl, cudaStream_t s) {
  ccm_context* ctx = pl->ctx;
  char* base = pl->d_arena;
  const Arena& ar = pl->ar;
  const UnitList& ul = pl->ul;
  // libraries and query orders for the timing launches
  CCM_CUDA(launch_order(reinterpret_cast<const float*>(base + ar.series),
                        reinterpret_cast<const OrderJob*>(base + ar.orders),
                        (int64_t)ul.orders.size(), ul.max_nm,
                        reinterpret_cast<int32_t*>(base + ar.order),
                        reinterpret_cast<unsigned long long*>(base + ar.order_scratch), s));
  CCM_CUDA(enqueue_obs(base, ar, ul, s));
  SamplerParams sp = sampler_params(base, ar);
  CCM_CUDA(launch_sampler(sp, 0, (int64_t)ul.units.size(), ul.max_nm, s));
  const int want = 6 * ctx->sm_count;
  WorkItem* d_items = nullptr;
  CCM_CUDA(cudaMallocAsync(&d_items, sizeof(WorkItem) * (size_t)want, s));
  cudaEvent_t e0, e1;
  CCM_CUDA(cudaEventCreate(&e0));
  CCM_CUDA(cudaEventCreate(&e1));
  ccm_status st = CCM_OK;
  for (int E = ul.emin; E <= ul.emax && st == CCM_OK; ++E) {
    if (pl->tuning.known[E]) continue;
    std::vector<WorkItem> all;
    for (const WorkItem& w : ul.items)
      if (ul.units[(size_t)w.unit].E == E) all.push_back(w);
    if ((int)all.size() < want) continue;
    std::vector<WorkItem> sample;  // evenly spaced over the cost-sorted list
    for (int q = 0; q < want; ++q) sample.push_back(all[(size_t)q * all.size() / (size_t)want]);
    cudaError_t ce = cudaMemcpyAsync(d_items, sample.data(), sizeof(WorkItem) * sample.size(),
                                     cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) { st = fail(CCM_ECUDA, cudaGetErrorString(ce)); break; }
    float best = 1e30f;
    int best_v = pl->tuning.variant[E], best_ma = pl->tuning.merge_at[E];
    for (int v = 0; v < 2; ++v)
      for (int ma : {1, 2, 4, 8}) {
        Tuning tn = pl->tuning;
        tn.variant[E] = v;
        tn.merge_at[E] = ma;
        KnnParams kp = knn_params(base, ar, ul, 0, tn);
        kp.items = d_items;
        kp.n_items = (int64_t)sample.size();
        float ms = 0.f;
        for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {  // warm-up, then timed
          ce = cudaEventRecord(e0, s);
          if (ce == cudaSuccess) ce = launch_knn(kp, E, (int)sample.size(), s);
          if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
          if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
          if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (ce != cudaSuccess) break;
        if (ms < best) {
          best = ms;
          best_v = v;
          best_ma = ma;
        }
      }
    if (ce != cudaSuccess) { st = fail(CCM_ECUDA, cudaGetErrorString(ce)); break; }
    pl->tuning.variant[E] = best_v;
    pl->tuning.merge_at[E] = best_ma;
    pl->tuning.known[E] = true;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      ctx->tuning.variant[E] = best_v;
      ctx->tuning.merge_at[E] = best_ma;
      ctx->tuning.known[E] = true;
    }
    save_cache(ctx, E, best_v, best_ma);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(d_items, s);
  if (st == CCM_OK) CCM_CUDA(cudaStreamSynchronize(s));
  return st;
}

}  // namespace

// ==================================================================== ABI ===
extern "C" {

const char* ccm_last_error(void) { return t_err.c_str(); }

const char* ccm_version(void) { return "ccm-gb300 0.1 (sm_103a)"; }

ccm_status ccm_context_create(int device, size_t hbm_budget_bytes, ccm_context** out) {
  if (!out) return fail(CCM_EINVAL, "out is NULL");
  *out = nullptr;
  int count = 0;
  CCM_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(CCM_EINVAL, "no such device");
  CCM_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  CCM_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major < 10) return fail(CCM_EINVAL, "needs a Blackwell (sm_10x) GPU");
  CCM_CUDA(sampler_prepare());
  CCM_CUDA(knn_prepare());
  CCM_CUDA(order_prepare());
  CCM_CUDA(table_prepare());
  CCM_CUDA(convergence_prepare());
  CCM_CUDA(knn_table_prepare());
  size_t free_b = 0, total_b = 0;
  CCM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  std::unique_ptr<ccm_context> ctx(new ccm_context());
  ctx->device = device;
  ctx->device_name = prop.name;
  ctx->sm_count = prop.multiProcessorCount;
  load_cache(ctx.get());
  if (const char* env = getenv("CCM_FAULT_INJECT_BATCH")) ctx->inject_batch = atoll(env);
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  *out = ctx.release();
  return CCM_OK;
}

ccm_status ccm_plan(ccm_context* ctx, const ccm_problem* prob, ccm_plan_t** out) {
  if (!ctx || !out) return fail(CCM_EINVAL, "NULL argument");
  *out = nullptr;
  std::unique_ptr<ccm_plan_s> pl(new ccm_plan_s());
  pl->ctx = ctx;
  ccm_status st = copy_problem(prob, &pl->pc);
  if (st != CCM_OK) return st;
  append_units(pl->pc, 0, 0, &pl->ul, table_cap(ctx));
  sort_items(&pl->ul);
  const int64_t series_elems = (int64_t)pl->pc.V * pl->pc.n;
  pl->ar = layout(series_elems, pl->ul, pl->ul.n_rho, pl->ul.max_nm);
  CCM_CUDA(cudaSetDevice(ctx->device));
  st = reserve(ctx, pl->ar.total);
  if (st != CCM_OK) return st;
  cudaError_t e = cudaMalloc(&pl->d_arena, pl->ar.total);
  if (e != cudaSuccess) {
    release(ctx, pl->ar.total);
    return fail(CCM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking);
  for (int q = 0; q < 5 && e == cudaSuccess; ++q) e = cudaEventCreate(&pl->ev[q]);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.units, pl->ul.units.data(),
                   sizeof(UnitDesc) * pl->ul.units.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.items, pl->ul.items.data(),
                   sizeof(WorkItem) * pl->ul.items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.orders, pl->ul.orders.data(),
                   sizeof(OrderJob) * pl->ul.orders.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.targets, pl->ul.targets.data(),
                   sizeof(TargetDesc) * pl->ul.targets.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.tables, pl->ul.tables.data(),
                   sizeof(TableJob) * pl->ul.tables.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.obs_jobs, pl->ul.obs_jobs.data(),
                   sizeof(ObsJob) * pl->ul.obs_jobs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_arena + pl->ar.items_table, pl->ul.items_table.data(),
                   sizeof(WorkItem) * pl->ul.items_table.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemset(pl->d_arena + pl->ar.done, 0, sizeof(uint32_t) * pl->ul.units.size());
  if (e != cudaSuccess) {
    cudaFree(pl->d_arena);
    if (pl->stream) cudaStreamDestroy(pl->stream);
    release(ctx, pl->ar.total);
    return fail(CCM_ECUDA, std::string("plan set-up: ") + cudaGetErrorString(e));
  }
  pl->grid = persistent_grid(ctx, pl->ul.emin, pl->ul.emax);
  {
    int per_sm = 1;
    if (knn_table_occupancy(pl->ul.max_nm, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    pl->grid_table = ctx->sm_count * per_sm;
  }
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    pl->tuning = ctx->tuning;
  }
  ccm_plan_info& in = pl->info;
  in.n_units = pl->ul.n_rho;
  in.n_queries = pl->ul.q_total;
  in.library_entries = pl->ul.lib_dbg_total;
  in.neighbour_entries = pl->ul.nbr_total;
  in.n_work_items = (int64_t)pl->ul.items.size();
  in.device_bytes = pl->ar.total;
  in.pair_count = pl->ul.pairs;
  in.flop_count = pl->ul.flops;
  in.brute_flop_count = pl->ul.brute_flops;
  in.brute_pair_count = pl->ul.brute_pairs;
  in.search_query_count = pl->ul.search_queries;
  in.table_query_count = pl->ul.table_queries;
  in.table_bytes = (pl->ul.table_elem() + sizeof(float) * (pl->ul.table_tv ? 2 : 1)) *
                   (size_t)pl->ul.table_total;
  // launches of one ccm_run: order, tables, sampler, one brute-force and one
  // table-scan kernel per E present
  in.launches_per_run = 3 + pl->ul.table_groups();  // order, observed moments, sampler, tables
  for (int E = 1; E <= kMaxE; ++E)
    in.launches_per_run += (pl->ul.e_count[E] > 0 ? 1 : 0) + (pl->ul.te_count[E] > 0 ? 1 : 0);
  *out = pl.release();
  return CCM_OK;
}

ccm_status ccm_plan_get_info(const ccm_plan_t* plan, ccm_plan_info* info) {
  if (!plan || !info) return fail(CCM_EINVAL, "NULL argument");
  *info = plan->info;
  return CCM_OK;
}

ccm_status ccm_plan_destroy(ccm_plan_t* plan) {
  if (!plan) return fail(CCM_EINVAL, "plan is NULL");
  cudaSetDevice(plan->ctx->device);
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  if (plan->stream) cudaStreamDestroy(plan->stream);
  for (cudaEvent_t ev : plan->ev)
    if (ev) cudaEventDestroy(ev);
  cudaFree(plan->d_arena);
  release(plan->ctx, plan->ar.total);
  delete plan;
  return CCM_OK;
}

ccm_status ccm_run_ex(ccm_plan_t* plan, const float* series, double* rho, const ccm_debug_out* dbg,
                      void* cuda_stream) {
  if (!plan || !series || !rho) return fail(CCM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(plan->run_mu);
  CCM_CUDA(cudaSetDevice(plan->ctx->device));
  const ProblemCopy& pc = plan->pc;
  const bool in_dev = (pc.flags & CCM_INPUT_ON_DEVICE) != 0;
  const bool out_dev = (pc.flags & CCM_OUTPUT_ON_DEVICE) != 0;
  const size_t series_bytes = sizeof(float) * (size_t)pc.V * (size_t)pc.n;
  if (!in_dev && !all_finite(series, (size_t)pc.V * (size_t)pc.n))
    return fail(CCM_EINVAL, "series holds a non-finite value");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : plan->stream;
  char* base = plan->d_arena;
  CCM_CUDA(cudaMemcpyAsync(base + plan->ar.series, series, series_bytes,
                           in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  const bool want_dbg = dbg && (dbg->libraries || dbg->neighbours || dbg->predictions);
  if (want_dbg) {
    // Checking path: direct launches with the per-unit outputs (no graph).
    const UnitList& ul = plan->ul;
    const size_t lb = sizeof(int32_t) * (size_t)ul.lib_dbg_total;
    const size_t nb = sizeof(int32_t) * (size_t)ul.nbr_total;
    const size_t xb = sizeof(float) * (size_t)ul.q_total;
    char* tmp = nullptr;
    if (!out_dev) {
      CCM_CUDA(cudaMallocAsync(&tmp, align_up(lb, 256) + align_up(nb, 256) + align_up(xb, 256), s));
    }
    int32_t* d_lib = dbg->libraries ? (out_dev ? dbg->libraries : reinterpret_cast<int32_t*>(tmp))
                                    : nullptr;
    int32_t* d_nbr = dbg->neighbours ? (out_dev ? dbg->neighbours
                                                : reinterpret_cast<int32_t*>(tmp + align_up(lb, 256)))
                                     : nullptr;
    float* d_xh = dbg->predictions
                      ? (out_dev ? dbg->predictions
                                 : reinterpret_cast<float*>(tmp + align_up(lb, 256) + align_up(nb, 256)))
                      : nullptr;
    ccm_status st =
        enqueue_sweep(base, plan->ar, ul, plan->tuning, plan->grid, plan->grid_table, 1, d_lib,
                      d_nbr, d_xh, s, plan->ev, false, (pc.flags & CCM_SEARCH_STATS) != 0);
    if (st != CCM_OK) return st;
    if (!out_dev) {
      if (dbg->libraries) CCM_CUDA(cudaMemcpyAsync(dbg->libraries, d_lib, lb, cudaMemcpyDeviceToHost, s));
      if (dbg->neighbours) CCM_CUDA(cudaMemcpyAsync(dbg->neighbours, d_nbr, nb, cudaMemcpyDeviceToHost, s));
      if (dbg->predictions) CCM_CUDA(cudaMemcpyAsync(dbg->predictions, d_xh, xb, cudaMemcpyDeviceToHost, s));
      CCM_CUDA(cudaFreeAsync(tmp, s));
    }
  } else {
    if (!plan->tuned) {
      bool missing = false;
      for (int e = plan->ul.emin; e <= plan->ul.emax; ++e)
        for (const int32_t E : pc.E) missing |= (E == e && !plan->tuning.known[e]);
      if (missing && !(pc.flags & CCM_NO_AUTOTUNE) && plan->ul.pairs >= kTunePairs) {
        ccm_status st = autotune(plan, s);
        if (st != CCM_OK) return st;
      }
      plan->tuned = true;
    }
    if (!plan->graph) {
      cudaGraph_t graph = nullptr;
      CCM_CUDA(cudaStreamBeginCapture(plan->stream, cudaStreamCaptureModeThreadLocal));
      ccm_status st = enqueue_sweep(base, plan->ar, plan->ul, plan->tuning, plan->grid,
                                    plan->grid_table, 1, nullptr, nullptr, nullptr, plan->stream,
                                    plan->ev, true, (pc.flags & CCM_SEARCH_STATS) != 0);
      const cudaError_t ce = cudaStreamEndCapture(plan->stream, &graph);
      if (st != CCM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      CCM_CUDA(ce);
      const cudaError_t ie = cudaGraphInstantiate(&plan->graph, graph, 0);
      cudaGraphDestroy(graph);
      CCM_CUDA(ie);
    }
    CCM_CUDA(cudaGraphLaunch(plan->graph, s));
  }
  const size_t rho_bytes = sizeof(double) * (size_t)plan->ul.n_rho;
  CCM_CUDA(cudaMemcpyAsync(rho, base + plan->ar.rho, rho_bytes,
                           out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!cuda_stream || !in_dev || !out_dev) return check_err_flag(base, plan->ar, s);
  return CCM_OK;
}

ccm_status ccm_plan_kernel_times(const ccm_plan_t* plan, double* sampler_ms, double* knn_ms) {
  double st[4];
  const ccm_status r = ccm_plan_stage_times(plan, st);
  if (r != CCM_OK) return r;
  if (sampler_ms) *sampler_ms = st[0] + st[1];
  if (knn_ms) *knn_ms = st[2] + st[3];
  return CCM_OK;
}

ccm_status ccm_plan_stage_times(const ccm_plan_t* plan, double* stage_ms) {
  if (!plan || !stage_ms) return fail(CCM_EINVAL, "NULL argument");
  CCM_CUDA(cudaSetDevice(plan->ctx->device));
  for (int q = 0; q < 4; ++q) {
    float t = 0.f;
    CCM_CUDA(cudaEventElapsedTime(&t, plan->ev[q], plan->ev[q + 1]));
    stage_ms[q] = t;
  }
  return CCM_OK;
}

ccm_status ccm_plan_search_stats(const ccm_plan_t* plan, ccm_search_stats* out) {
  if (!plan || !out) return fail(CCM_EINVAL, "NULL argument");
  if (!(plan->pc.flags & CCM_SEARCH_STATS))
    return fail(CCM_EINVAL, "the plan was made without CCM_SEARCH_STATS");
  CCM_CUDA(cudaSetDevice(plan->ctx->device));
  unsigned long long c[kStatCount];
  CCM_CUDA(cudaMemcpy(c, plan->d_arena + plan->ar.stats, sizeof(c), cudaMemcpyDeviceToHost));
  out->brute_tiles = c[kStatBruteTiles];
  out->brute_queries = c[kStatBruteQueries];
  out->pairs_begun = c[kStatPairsBegun];
  out->pairs_full = c[kStatPairsFull];
  out->pairs_pruned = c[kStatPairsPruned];
  out->candidates = c[kStatCandidates];
  out->merge_slots = c[kStatMergeSlots];
  out->table_queries = c[kStatTableQueries];
  out->table_entries = c[kStatTableEntries];
  out->table_fallbacks = c[kStatTableFallbacks];
  return CCM_OK;
}

ccm_status ccm_run(ccm_plan_t* plan, const float* series, double* rho, void* cuda_stream) {
  return ccm_run_ex(plan, series, rho, nullptr, cuda_stream);
}

ccm_status ccm_run_plain(ccm_plan_t* plan, const float* series, double* rho, void* cuda_stream) {
  if (!plan || !series || !rho) return fail(CCM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(plan->run_mu);
  CCM_CUDA(cudaSetDevice(plan->ctx->device));
  const ProblemCopy& pc = plan->pc;
  const bool in_dev = (pc.flags & CCM_INPUT_ON_DEVICE) != 0;
  const bool out_dev = (pc.flags & CCM_OUTPUT_ON_DEVICE) != 0;
  if (!in_dev && !all_finite(series, (size_t)pc.V * (size_t)pc.n))
    return fail(CCM_EINVAL, "series holds a non-finite value");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : plan->stream;
  char* base = plan->d_arena;
  const Arena& ar = plan->ar;
  CCM_CUDA(cudaMemcpyAsync(base + ar.series, series, sizeof(float) * (size_t)pc.V * (size_t)pc.n,
                           in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CCM_CUDA(cudaMemsetAsync(base + ar.err, 0, sizeof(int32_t), s));
  const SamplerParams sp = sampler_params(base, ar);
  const UnitDesc* d_units = reinterpret_cast<const UnitDesc*>(base + ar.units);
  const TargetDesc* d_targets = reinterpret_cast<const TargetDesc*>(base + ar.targets);
  CCM_CUDA(launch_order(reinterpret_cast<const float*>(base + ar.series),
                        reinterpret_cast<const OrderJob*>(base + ar.orders),
                        (int64_t)plan->ul.orders.size(), plan->ul.max_nm,
                        reinterpret_cast<int32_t*>(base + ar.order),
                        reinterpret_cast<unsigned long long*>(base + ar.order_scratch), s));
  for (size_t q = 0; q < plan->ul.units.size(); ++q) {
    const UnitDesc& u = plan->ul.units[q];
    CCM_CUDA(launch_sampler(sp, (int64_t)q, 1, u.n_m, s));
    for (int32_t t = 0; t < u.n_targets; ++t)
      CCM_CUDA(launch_plain_unit(reinterpret_cast<const float*>(base + ar.series), d_units + q, u,
                                 d_targets + u.tgt_off + t,
                                 reinterpret_cast<const int32_t*>(base + ar.lib),
                                 reinterpret_cast<float*>(base + ar.scratch),
                                 reinterpret_cast<double*>(base + ar.rho), s));
  }
  CCM_CUDA(cudaMemcpyAsync(rho, base + ar.rho, sizeof(double) * (size_t)plan->ul.n_rho,
                           out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!cuda_stream || !in_dev || !out_dev) return check_err_flag(base, ar, s);
  return CCM_OK;
}

ccm_status ccm_convergence(ccm_context* ctx, const double* rho, int64_t n_rows, int32_t n_L,
                           const int64_t* L, int32_t r, double z_crit,
                           ccm_convergence_t* out, uint32_t flags, void* cuda_stream) {
  static_assert(sizeof(ConvergenceRow) == sizeof(ccm_convergence_t), "layout");
  if (!ctx || !rho || !L || !out) return fail(CCM_EINVAL, "NULL argument");
  if (n_rows < 0 || n_rows > 0x7fffffff) return fail(CCM_EINVAL, "n_rows out of range");
  if (n_L < 2 || n_L > kMaxConvGroups) return fail(CCM_EINVAL, "n_L must be in 2..64");
  if (r < 1 || (int64_t)n_L * r > kMaxConvValues)
    return fail(CCM_EINVAL, "need r >= 1 and n_L*r <= 24576");
  if (std::isnan(z_crit)) return fail(CCM_EINVAL, "z_crit is NaN");
  ConvOrder ord;
  std::memset(&ord, 0, sizeof(ord));
  for (int32_t g = 0; g < n_L; ++g) ord.group[g] = g;
  std::stable_sort(ord.group, ord.group + n_L, [&](int32_t a, int32_t b) { return L[a] < L[b]; });
  for (int32_t g = 1; g < n_L; ++g)
    if (L[ord.group[g]] == L[ord.group[g - 1]]) return fail(CCM_EINVAL, "L values must differ");
  if (n_rows == 0) return CCM_OK;
  CCM_CUDA(cudaSetDevice(ctx->device));
  const bool in_dev = (flags & CCM_INPUT_ON_DEVICE) != 0;
  const bool out_dev = (flags & CCM_OUTPUT_ON_DEVICE) != 0;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t rho_bytes = sizeof(double) * (size_t)n_rows * (size_t)n_L * (size_t)r;
  const size_t out_bytes = sizeof(ccm_convergence_t) * (size_t)n_rows;
  double* d_rho = const_cast<double*>(rho);
  ConvergenceRow* d_out = reinterpret_cast<ConvergenceRow*>(out);
  void* tmp = nullptr;
  if (!in_dev || !out_dev) {
    CCM_CUDA(cudaMalloc(&tmp, (in_dev ? 0 : rho_bytes + 256) + (out_dev ? 0 : out_bytes)));
    char* t = static_cast<char*>(tmp);
    if (!in_dev) {
      d_rho = reinterpret_cast<double*>(t);
      t += (rho_bytes + 255) / 256 * 256;
    }
    if (!out_dev) d_out = reinterpret_cast<ConvergenceRow*>(t);
  }
  cudaError_t e = cudaSuccess;
  if (!in_dev) e = cudaMemcpyAsync(d_rho, rho, rho_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_convergence(d_rho, n_rows, n_L, r, ord, z_crit, d_out, s);
  if (e == cudaSuccess && !out_dev)
    e = cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && (tmp || !cuda_stream)) e = cudaStreamSynchronize(s);
  if (tmp) {
    const cudaError_t e2 = cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return fail(CCM_ECUDA, std::string("ccm_convergence: ") + cudaGetErrorString(e));
  return CCM_OK;
}

}  // extern "C"

// ================================================================ serving ===
struct Job {
  uint64_t ticket = 0;
  ProblemCopy pc;
  float* h_series = nullptr;  // pinned copy (from the context's pool)
  double* h_rho = nullptr;    // pinned result (from the context's pool)
  size_t series_bytes = 0, rho_bytes = 0;
  int64_t n_units = 0;
  size_t footprint = 0;
  double pairs = 0.0;  // query-library pairs: the job's cost
  enum State { kQueued, kRunning, kDone, kFailed, kCancelled } state = kQueued;
  ccm_status status = CCM_PENDING;
  std::string err;
  double t_submit = 0, t_start = 0, t_finish = 0;
};

struct Batch {
  ccm_context* ctx = nullptr;
  std::vector<std::shared_ptr<Job>> jobs;
  UnitList ul;
  Arena ar;
  char* d_arena = nullptr;
  int32_t* h_err = nullptr;
  void* h_meta = nullptr;  // pinned copy of units, items and order jobs for the async upload
  size_t meta_bytes = 0;
  cudaStream_t stream = nullptr;
  std::atomic<bool> finished{false};
};

namespace {

size_t job_footprint(const ccm_context* ctx, const ProblemCopy& pc, double* pairs) {
  UnitList ul;
  append_units(pc, 0, 0, &ul, table_cap(ctx));
  *pairs = ul.pairs;
  return layout((int64_t)pc.V * pc.n, ul, ul.n_rho, 0).total;
}

void CUDART_CB on_batch_done(void* arg) {
  Batch* b = static_cast<Batch*>(arg);
  ccm_context* ctx = b->ctx;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    b->finished.store(true);
  }
  ctx->cv.notify_all();
}

// Launch one batch (called by the serving thread without ctx->mu held).
// `inject`: the fault-injection hook chose this batch; it fails after its
// arena and series uploads have been enqueued, like a failing CUDA call there.
ccm_status launch_batch(ccm_context* ctx, Batch* b, bool inject) {
  int64_t series_elems = 0, out = 0;
  for (auto& j : b->jobs) {
    append_units(j->pc, series_elems, out, &b->ul, table_cap(ctx));
    series_elems += (int64_t)j->pc.V * j->pc.n;
    out += j->n_units;
  }
  sort_items(&b->ul);
  b->ar = layout(series_elems, b->ul, out, 0);
  CCM_CUDA(cudaMallocAsync(&b->d_arena, b->ar.total, b->stream));
  char* base = b->d_arena;
  int64_t so = 0;
  for (auto& j : b->jobs) {
    const size_t bytes = sizeof(float) * (size_t)j->pc.V * (size_t)j->pc.n;
    CCM_CUDA(cudaMemcpyAsync(base + b->ar.series + sizeof(float) * so, j->h_series, bytes,
                             cudaMemcpyHostToDevice, b->stream));
    so += (int64_t)j->pc.V * j->pc.n;
  }
  if (inject) return fail(CCM_ECUDA, "injected fault (CCM_FAULT_INJECT_BATCH): batch launch failed");
  // Descriptors go through pinned staging: a copy from pageable memory would
  // wait for earlier work on this (reused) stream.
  // (units, work items, order jobs, targets, table jobs, table work items,
  // observed-moment jobs)
  constexpr int kMeta = 7;
  const void* src[kMeta] = {b->ul.units.data(),   b->ul.items.data(),  b->ul.orders.data(),
                            b->ul.targets.data(), b->ul.tables.data(), b->ul.items_table.data(),
                            b->ul.obs_jobs.data()};
  const size_t len[kMeta] = {sizeof(UnitDesc) * b->ul.units.size(),
                             sizeof(WorkItem) * b->ul.items.size(),
                             sizeof(OrderJob) * b->ul.orders.size(),
                             sizeof(TargetDesc) * b->ul.targets.size(),
                             sizeof(TableJob) * b->ul.tables.size(),
                             sizeof(WorkItem) * b->ul.items_table.size(),
                             sizeof(ObsJob) * b->ul.obs_jobs.size()};
  const size_t dst[kMeta] = {b->ar.units,  b->ar.items,       b->ar.orders,  b->ar.targets,
                             b->ar.tables, b->ar.items_table, b->ar.obs_jobs};
  b->meta_bytes = 0;
  for (int q = 0; q < kMeta; ++q) b->meta_bytes += len[q];
  b->h_meta = pinned_get(ctx, b->meta_bytes);
  if (!b->h_meta) return fail(CCM_ENOMEM, "pinned allocation failed");
  char* hm = static_cast<char*>(b->h_meta);
  for (int q = 0; q < kMeta; ++q) {
    if (len[q] == 0) continue;
    std::memcpy(hm, src[q], len[q]);
    CCM_CUDA(cudaMemcpyAsync(base + dst[q], hm, len[q], cudaMemcpyHostToDevice, b->stream));
    hm += len[q];
  }
  CCM_CUDA(cudaMemsetAsync(base + b->ar.done, 0, sizeof(uint32_t) * b->ul.units.size(), b->stream));
  Tuning tn;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    tn = ctx->tuning;
  }
  ccm_status st =
      enqueue_sweep(base, b->ar, b->ul, tn, 0, 0, 0, nullptr, nullptr, nullptr, b->stream);
  if (st != CCM_OK) return st;
  int64_t ro = 0;
  for (auto& j : b->jobs) {
    CCM_CUDA(cudaMemcpyAsync(j->h_rho, base + b->ar.rho + sizeof(double) * ro,
                             sizeof(double) * (size_t)j->n_units, cudaMemcpyDeviceToHost, b->stream));
    ro += j->n_units;
  }
  CCM_CUDA(cudaMemcpyAsync(b->h_err, base + b->ar.err, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           b->stream));
  CCM_CUDA(cudaFreeAsync(b->d_arena, b->stream));
  b->d_arena = nullptr;  // freed in stream order: the error path must not free it again
  CCM_CUDA(cudaLaunchHostFunc(b->stream, on_batch_done, b));
  return CCM_OK;
}

// No CUDA call that may synchronise (cudaFreeHost, cudaMallocHost,
// cudaStreamSynchronize, ...) is made while ctx->mu is held: the host callback
// that marks a batch finished takes ctx->mu, and its stream cannot advance
// until it returns.
void serve(ccm_context* ctx) {
  cudaSetDevice(ctx->device);
  std::vector<int32_t*> to_free;
  std::unique_lock<std::mutex> lk(ctx->mu);
  for (;;) {
    // Retire finished batches.
    for (auto it = ctx->inflight.begin(); it != ctx->inflight.end();) {
      Batch* b = it->get();
      if (!b->finished.load()) {
        ++it;
        continue;
      }
      const double t = now_s();
      size_t bytes = 0;
      for (auto& j : b->jobs) {
        bytes += j->footprint;
        j->t_finish = t;
        if (*b->h_err != 0) {
          j->state = Job::kFailed;
          j->status = CCM_ECUDA;
          j->err = "kernel reported error flag " + std::to_string(*b->h_err);
        } else {
          j->state = Job::kDone;
          j->status = CCM_OK;
        }
      }
      ctx->used -= std::min(ctx->used, bytes);
      // cudaFreeHost may synchronise; a pending host callback of another batch
      // needs ctx->mu to finish, so free after releasing the lock.
      to_free.push_back(b->h_err);
      pinned_put(ctx, b->h_meta, b->meta_bytes);  // pool mutex only, no CUDA call
      it = ctx->inflight.erase(it);
      ctx->cv.notify_all();
    }
    if (!to_free.empty()) {
      lk.unlock();
      for (int32_t* ptr : to_free) pinned_put(ctx, ptr, sizeof(int32_t));
      to_free.clear();
      lk.lock();
      continue;  // state may have changed while unlocked
    }
    if (ctx->stop && ctx->inflight.empty()) break;
    // Admit queued jobs into a new batch while their footprints fit.
    if (!ctx->stop && !ctx->queue.empty() && (int)ctx->inflight.size() < ctx->max_inflight) {
      auto b = std::make_shared<Batch>();
      b->ctx = ctx;
      size_t bytes = 0;
      int64_t units = 0;
      double pairs = 0.0;
      // A batch takes queued jobs in order while they fit the free budget; a
      // large job runs alone, small ones are grouped up to batch_pairs.
      while (!ctx->queue.empty()) {
        auto& j = ctx->queue.front();
        if (j->state == Job::kCancelled) {
          ctx->queue.pop_front();
          continue;
        }
        if (ctx->used + bytes + j->footprint > ctx->budget) break;
        if (!b->jobs.empty() && (units + j->n_units > (int64_t)1 << 22 ||
                                 pairs + j->pairs > ctx->batch_pairs))
          break;
        bytes += j->footprint;
        units += j->n_units;
        pairs += j->pairs;
        b->jobs.push_back(j);
        ctx->queue.pop_front();
      }
      if (!b->jobs.empty()) {
        ctx->used += bytes;
        const double t = now_s();
        for (auto& j : b->jobs) {
          j->state = Job::kRunning;
          j->t_start = t;
        }
        b->stream = (pairs <= ctx->batch_pairs)
                        ? ctx->fast_streams[ctx->next_fast++ % ctx->fast_streams.size()]
                        : ctx->streams[ctx->next_stream++ % ctx->streams.size()];
        ctx->inflight.push_back(b);
        const bool inject = ctx->batches_launched++ == ctx->inject_batch;
        lk.unlock();
        b->h_err = static_cast<int32_t*>(pinned_get(ctx, sizeof(int32_t)));
        ccm_status st = b->h_err ? launch_batch(ctx, b.get(), inject)
                                 : fail(CCM_ENOMEM, "pinned allocation failed");
        lk.lock();
        if (st != CCM_OK) {
          // Nothing more will run for this batch once the stream drains.
          lk.unlock();
          cudaStreamSynchronize(b->stream);
          if (b->d_arena) cudaFree(b->d_arena);
          lk.lock();
          for (auto& j : b->jobs) {
            j->state = Job::kFailed;
            j->status = st;
            j->err = t_err;
            j->t_finish = now_s();
          }
          ctx->used -= std::min(ctx->used, bytes);
          if (b->h_err) to_free.push_back(b->h_err);
          pinned_put(ctx, b->h_meta, b->meta_bytes);
          ctx->inflight.remove(b);
          ctx->cv.notify_all();
        }
        continue;
      }
    }
    ctx->cv.wait_for(lk, std::chrono::milliseconds(50));
  }
}

ccm_status ensure_server(ccm_context* ctx) {
  std::lock_guard<std::mutex> g(ctx->mu);
  if (ctx->server_started) return CCM_OK;
  int least = 0, greatest = 0;
  CCM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  for (int q = 0; q < ctx->max_inflight / 2; ++q) {
    cudaStream_t s;
    CCM_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, least));
    ctx->streams.push_back(s);
    CCM_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest));
    ctx->fast_streams.push_back(s);
  }
  ctx->server = std::thread(serve, ctx);
  ctx->server_started = true;
  return CCM_OK;
}

void free_job(ccm_context* ctx, Job* j) {
  pinned_put(ctx, j->h_series, j->series_bytes);
  pinned_put(ctx, j->h_rho, j->rho_bytes);
  j->h_series = nullptr;
  j->h_rho = nullptr;
}

}  // namespace

extern "C" {

ccm_status ccm_submit(ccm_context* ctx, const ccm_problem* prob, const float* series,
                      uint64_t* ticket) {
  if (!ctx || !series || !ticket) return fail(CCM_EINVAL, "NULL argument");
  auto j = std::make_shared<Job>();
  ccm_status st = copy_problem(prob, &j->pc);
  if (st != CCM_OK) return st;
  if (j->pc.flags & (CCM_INPUT_ON_DEVICE | CCM_OUTPUT_ON_DEVICE))
    return fail(CCM_EINVAL, "ccm_submit takes host series and returns host rho");
  const size_t elems = (size_t)j->pc.V * (size_t)j->pc.n;
  if (!all_finite(series, elems)) return fail(CCM_EINVAL, "series holds a non-finite value");
  j->n_units = j->pc.n_units();
  j->footprint = job_footprint(ctx, j->pc, &j->pairs);
  if (j->footprint > ctx->budget)
    return fail(CCM_ETOOLARGE, "job footprint " + std::to_string(j->footprint) +
                                   " B exceeds the context budget");
  CCM_CUDA(cudaSetDevice(ctx->device));
  st = ensure_server(ctx);
  if (st != CCM_OK) return st;
  j->series_bytes = sizeof(float) * elems;
  j->rho_bytes = sizeof(double) * (size_t)j->n_units;
  j->h_series = static_cast<float*>(pinned_get(ctx, j->series_bytes));
  j->h_rho = static_cast<double*>(pinned_get(ctx, j->rho_bytes));
  if (!j->h_series || !j->h_rho) {
    free_job(ctx, j.get());
    return fail(CCM_ENOMEM, "pinned allocation failed");
  }
  std::memcpy(j->h_series, series, sizeof(float) * elems);
  j->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    j->ticket = ctx->next_ticket++;
    ctx->jobs[j->ticket] = j;
    ctx->queue.push_back(j);
  }
  ctx->cv.notify_all();
  *ticket = j->ticket;
  return CCM_OK;
}

ccm_status ccm_poll(ccm_context* ctx, uint64_t ticket, double* rho, int32_t timeout_ms) {
  if (!ctx) return fail(CCM_EINVAL, "context is NULL");
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto it = ctx->jobs.find(ticket);
  if (it == ctx->jobs.end()) return fail(CCM_ENOTFOUND, "unknown ticket");
  std::shared_ptr<Job> j = it->second;
  auto finished = [&] {
    return j->state == Job::kDone || j->state == Job::kFailed || j->state == Job::kCancelled;
  };
  if (!finished() && timeout_ms > 0)
    ctx->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
  if (!finished()) return CCM_PENDING;
  ccm_status st = j->status;
  if (j->state == Job::kDone) {
    if (!rho) return fail(CCM_EINVAL, "rho is NULL");
    std::memcpy(rho, j->h_rho, sizeof(double) * (size_t)j->n_units);
  } else {
    t_err = j->err;
  }
  ctx->jobs.erase(it);
  lk.unlock();
  free_job(ctx, j.get());
  return st;
}

ccm_status ccm_cancel(ccm_context* ctx, uint64_t ticket) {
  if (!ctx) return fail(CCM_EINVAL, "context is NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->jobs.find(ticket);
  if (it == ctx->jobs.end()) return fail(CCM_ENOTFOUND, "unknown ticket");
  Job* j = it->second.get();
  if (j->state != Job::kQueued) return CCM_PENDING;
  j->state = Job::kCancelled;
  j->status = CCM_ECANCELLED;
  j->err = "cancelled";
  j->t_finish = now_s();
  ctx->cv.notify_all();
  return CCM_OK;
}

ccm_status ccm_job_times(ccm_context* ctx, uint64_t ticket, double* submit_s, double* start_s,
                         double* finish_s) {
  if (!ctx) return fail(CCM_EINVAL, "context is NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->jobs.find(ticket);
  if (it == ctx->jobs.end()) return fail(CCM_ENOTFOUND, "unknown ticket");
  Job* j = it->second.get();
  if (submit_s) *submit_s = j->t_submit;
  if (start_s) *start_s = j->t_start;
  if (finish_s) *finish_s = j->t_finish;
  return (j->state == Job::kDone || j->state == Job::kFailed || j->state == Job::kCancelled)
             ? CCM_OK
             : CCM_PENDING;
}

ccm_status ccm_context_destroy(ccm_context* ctx) {
  if (!ctx) return fail(CCM_EINVAL, "context is NULL");
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->stop = true;
    for (auto& j : ctx->queue) {
      if (j->state == Job::kQueued) {
        j->state = Job::kCancelled;
        j->status = CCM_ECANCELLED;
      }
    }
    ctx->queue.clear();
  }
  ctx->cv.notify_all();
  if (ctx->server_started) ctx->server.join();
  cudaSetDevice(ctx->device);
  for (cudaStream_t s : ctx->streams) cudaStreamDestroy(s);
  for (cudaStream_t s : ctx->fast_streams) cudaStreamDestroy(s);
  for (auto& kv : ctx->jobs) free_job(ctx, kv.second.get());
  ctx->jobs.clear();
  for (void* ptr : ctx->pool_all) cudaFreeHost(ptr);
  delete ctx;
  return CCM_OK;
}

}  // extern "C"
