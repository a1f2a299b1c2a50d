// ccm_run_noalloc: one CCM cell without any device allocation.
//
// Some callers cannot call cudaMalloc at run time: a host framework whose own
// caching allocator already owns the device memory (a second allocator would
// fail or fragment it), or a latency-critical loop where cudaMalloc/cudaFree
// may synchronise the device implicitly.  For them this entry point computes
// one (pair, E, tau, L) cell with r realizations from caller-owned device
// input to caller-owned device output, and keeps every intermediate -- the
// realization descriptors, the work items, the r libraries, the per-tile
// partial moments, the observed-value tile records and the counters -- in one
// file-scope device array of
// kScratchBytes.  The array exists on every GPU that loads this library until
// the process exits.
//
// Set-up: the first call on a device (with that device current) sets the
// kernels' shared-memory attributes and looks the array's device address up
// with cudaGetSymbolAddress; later calls on that device reuse the address.
// Make that first call before any stream capture.
//
// Sharing: every call uses the same array, which keeps the previous call's
// contents; a set-up kernel at the start of each call rewrites the
// descriptors and clears the counters that must start at zero.  Calls whose
// work overlaps on the GPU (different streams, or several host threads)
// race on the array and give wrong results: serialise them.
#include <mutex>
#include <string>

#include "ccm.h"
#include "ccm_internal.h"

namespace ccm {

// Scratch for one cell: descriptors, work items, libraries, partial moments,
// counters, query order, observed-value tile records.  16 MiB holds, e.g., r = 250 realizations of L = 9000 at N = 10^4.
constexpr size_t kScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

struct NoallocLayout {
  size_t units, items, lib, part, done, err, counter, order, orderjob, target, obs, obsjob, total;
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

NoallocLayout noalloc_layout(int64_t r, int64_t L, int64_t n_tiles, int64_t n_m) {
  NoallocLayout a;
  size_t o = 0;
  a.units = o;
  o = up256(o + sizeof(UnitDesc) * (size_t)r);
  a.items = o;
  o = up256(o + sizeof(WorkItem) * (size_t)(r * n_tiles));
  a.lib = o;
  o = up256(o + sizeof(int32_t) * (size_t)(r * L));
  a.part = o;
  o = up256(o + 6 * sizeof(double) * (size_t)(r * n_tiles));
  a.done = o;
  o = up256(o + sizeof(uint32_t) * (size_t)r);
  a.err = o;
  o = up256(o + sizeof(int32_t));
  a.counter = o;
  o = up256(o + sizeof(uint32_t));
  a.order = o;
  o = up256(o + sizeof(int32_t) * (size_t)n_m);
  a.orderjob = o;
  o = up256(o + sizeof(OrderJob));
  a.target = o;
  o = up256(o + sizeof(TargetDesc) * (size_t)r);
  a.obs = o;
  o = up256(o + sizeof(double) * kObsStride * (size_t)n_tiles);
  a.obsjob = o;
  o = up256(o + sizeof(ObsJob));
  a.total = o;
  return a;
}

struct CellArgs {
  int64_t n;
  uint64_t seed;
  int32_t j, i, E, tau, L, r, n_m, n_tiles;
};

// Writes the descriptors and work items of the cell into the scratch and
// clears the counters and the error flag.
__global__ void noalloc_setup_kernel(unsigned char* scratch, NoallocLayout lay, CellArgs c) {
  UnitDesc* units = reinterpret_cast<UnitDesc*>(scratch + lay.units);
  WorkItem* items = reinterpret_cast<WorkItem*>(scratch + lay.items);
  uint32_t* done = reinterpret_cast<uint32_t*>(scratch + lay.done);
  const int64_t per_unit = (c.n_tiles + kBruteChunk - 1) / kBruteChunk;  // items per realization
  const int64_t n_items = (int64_t)c.r * per_unit;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_items;
       w += (int64_t)gridDim.x * blockDim.x) {
    items[w].unit = (int32_t)(w / per_unit);
    items[w].tile = (int32_t)((w % per_unit) * kBruteChunk);
    items[w].count = 1;
  }
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < c.r;
       k += (int64_t)gridDim.x * blockDim.x) {
    UnitDesc u;
    u.series_off = 0;
    u.n = c.n;
    u.lib_off = k * (int64_t)c.L;
    u.part_off = k * (int64_t)c.n_tiles;
    u.order_off = 0;
    u.tgt_off = k;
    u.seed = c.seed;
    u.j = c.j;
    u.E = c.E;
    u.tau = c.tau;
    u.L = c.L;
    u.k = (int32_t)k;
    u.n_m = c.n_m;
    u.n_tiles = c.n_tiles;
    u.n_targets = 1;
    u.table_off = 0;
    u.table_R = 0;
    u.theiler = 0;
    u.wfloor = 0.f;
    u.table_tv = 0;
    TargetDesc tg;
    tg.out_idx = k;
    tg.q_off = k * (int64_t)c.n_m;
    tg.nbr_off = k * (int64_t)c.n_m * (c.E + 1);
    tg.lib_dbg_off = k * (int64_t)c.L;
    tg.obs_tile = 0;
    tg.i = c.i;
    tg.pad = 0;
    reinterpret_cast<TargetDesc*>(scratch + lay.target)[k] = tg;
    units[k] = u;
    done[k] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    OrderJob oj;
    oj.series_off = 0;
    oj.n = c.n;
    oj.order_off = 0;
    oj.scratch_off = -1;  // long manifolds keep time order here (no scratch)
    oj.j = c.j;
    oj.E = c.E;
    oj.tau = c.tau;
    oj.n_m = c.n_m;
    *reinterpret_cast<OrderJob*>(scratch + lay.orderjob) = oj;
    ObsJob ob;
    ob.series_off = 0;
    ob.n = c.n;
    ob.order_off = 0;
    ob.obs_tile = 0;
    ob.i = c.i;
    ob.E = c.E;
    ob.tau = c.tau;
    ob.n_m = c.n_m;
    ob.n_tiles = c.n_tiles;
    ob.pad = 0;
    *reinterpret_cast<ObsJob*>(scratch + lay.obsjob) = ob;
    *reinterpret_cast<int32_t*>(scratch + lay.err) = 0;
    *reinterpret_cast<uint32_t*>(scratch + lay.counter) = 0u;
  }
}

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[64] = {nullptr};  // per device, found at first use

ccm_status noalloc_fail(ccm_status st, const std::string& msg) {
  set_last_error(msg.c_str());  // read back with ccm_last_error()
  return st;
}

}  // namespace
}  // namespace ccm

using namespace ccm;

extern "C" ccm_status ccm_run_noalloc(const float* d_series, int32_t n_series, int64_t n,
                                      int32_t j, int32_t i, int32_t E, int32_t tau, int64_t L,
                                      int32_t r, uint64_t seed, double* d_rho,
                                      void* cuda_stream) {
  if (!d_series || !d_rho) return noalloc_fail(CCM_EINVAL, "NULL series or rho");
  if (n_series < 2 || j < 0 || j >= n_series || i < 0 || i >= n_series || i == j)
    return noalloc_fail(CCM_EINVAL, "invalid pair (need 0 <= i, j < n_series, i != j)");
  if (E < 1 || E > kMaxE) return noalloc_fail(CCM_EINVAL, "E must be in 1..10");
  if (tau < 1) return noalloc_fail(CCM_EINVAL, "tau must be >= 1");
  if (n < 3 || n > 0x7fffffff) return noalloc_fail(CCM_EINVAL, "series length out of range");
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  if (L < E + 2 || L > n_m) return noalloc_fail(CCM_EINVAL, "L outside [E+2, N_m]");
  if (r < 1) return noalloc_fail(CCM_EINVAL, "r must be >= 1");
  const int64_t tileq = (int64_t)knn_block_threads() * knn_queries_per_thread();
  const int64_t n_tiles = (n_m + tileq - 1) / tileq;
  const NoallocLayout lay = noalloc_layout(r, L, n_tiles, n_m);
  if (lay.total > kScratchBytes)
    return noalloc_fail(CCM_ETOOLARGE,
                        "cell needs " + std::to_string(lay.total) + " B of scratch; the fixed "
                        "array holds " + std::to_string(kScratchBytes) + " B (reduce r or L)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(CCM_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return noalloc_fail(CCM_EINVAL, "device index out of range");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      e = sampler_prepare();
      if (e == cudaSuccess) e = knn_prepare();
      if (e == cudaSuccess) e = order_prepare();
      void* p = nullptr;
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(CCM_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CellArgs c;
  c.n = n;
  c.seed = seed;
  c.j = j;
  c.i = i;
  c.E = E;
  c.tau = tau;
  c.L = (int32_t)L;
  c.r = r;
  c.n_m = (int32_t)n_m;
  c.n_tiles = (int32_t)n_tiles;
  noalloc_setup_kernel<<<(unsigned)((r * n_tiles + 255) / 256), 256, 0, s>>>(scratch, lay, c);
  e = launch_order(d_series, reinterpret_cast<const OrderJob*>(scratch + lay.orderjob), 1,
                   (int)n_m, reinterpret_cast<int32_t*>(scratch + lay.order), nullptr, s);
  if (e == cudaSuccess)
    e = launch_obs(d_series, reinterpret_cast<const int32_t*>(scratch + lay.order),
                   reinterpret_cast<const ObsJob*>(scratch + lay.obsjob), 1, n_tiles,
                   reinterpret_cast<double*>(scratch + lay.obs), s);
  if (e != cudaSuccess) return noalloc_fail(CCM_ECUDA, cudaGetErrorString(e));
  SamplerParams sp{};
  sp.units = reinterpret_cast<const UnitDesc*>(scratch + lay.units);
  sp.targets = reinterpret_cast<const TargetDesc*>(scratch + lay.target);
  sp.order = reinterpret_cast<const int32_t*>(scratch + lay.order);
  sp.lib = reinterpret_cast<int32_t*>(scratch + lay.lib);
  sp.err = reinterpret_cast<int32_t*>(scratch + lay.err);
  e = launch_sampler(sp, 0, r, (int)n_m, s);
  if (e != cudaSuccess) return noalloc_fail(CCM_ECUDA, cudaGetErrorString(e));
  KnnParams kp{};
  kp.series = d_series;
  kp.units = reinterpret_cast<const UnitDesc*>(scratch + lay.units);
  kp.targets = reinterpret_cast<const TargetDesc*>(scratch + lay.target);
  kp.items = reinterpret_cast<const WorkItem*>(scratch + lay.items);
  kp.n_items = (int64_t)r * ((n_tiles + kBruteChunk - 1) / kBruteChunk);
  kp.lib = reinterpret_cast<const int32_t*>(scratch + lay.lib);
  kp.order = reinterpret_cast<const int32_t*>(scratch + lay.order);
  kp.partials = reinterpret_cast<double*>(scratch + lay.part);
  kp.obs = reinterpret_cast<const double*>(scratch + lay.obs);
  kp.unit_done = reinterpret_cast<uint32_t*>(scratch + lay.done);
  kp.item_counter = reinterpret_cast<uint32_t*>(scratch + lay.counter);
  kp.rho = d_rho;
  kp.err = reinterpret_cast<int32_t*>(scratch + lay.err);
  kp.persistent = 0;
  for (int q = 0; q <= kMaxE; ++q) {
    kp.merge_at[q] = kDefaultMergeAt;
    kp.variant[q] = kDefaultVariant;
  }
  e = launch_knn(kp, E, (int)kp.n_items, s);
  if (e != cudaSuccess) return noalloc_fail(CCM_ECUDA, cudaGetErrorString(e));
  if (!cuda_stream) {
    int32_t err = 0;
    e = cudaMemcpyAsync(&err, scratch + lay.err, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(CCM_ECUDA, cudaGetErrorString(e));
    if (err != 0)
      return noalloc_fail(CCM_ECUDA, "kernel reported error flag " + std::to_string(err));
  }
  return CCM_OK;
}
