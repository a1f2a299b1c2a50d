// Fused nearest-neighbour search + simplex projection + skill moments.
//
// For one query tile of one realization (paper Sect. 3.2: "finding the E+1
// nearest neighbors for every lagged-coordinate vector", the step the paper
// names as the most time-consuming), every query point of the shadow manifold
// M_j is compared with every library point; the E+1 nearest (itself
// excluded) give the simplex prediction of the target variable (Sect. 2.1),
// and the tile's FP64 moments of (observed, predicted) are merged per
// realization into the Pearson skill (Sect. 2.1).
//
// Design (GB300, FP32 on the CUDA cores; E <= 10 is not a dense contraction):
//  * persistent CTAs pull work items, sorted by cost, from an atomic counter;
//    a brute-force item is up to eight query tiles of one realization, so a
//    library that fits one shared-memory tile is staged once for all of them;
//  * each thread owns one query; library points sit in shared memory in
//    pairs, packed {a_e, b_e} per coordinate, so one sub.f32x2 + fma.f32x2
//    pair advances the query's distances to two points;
//  * a broadcast 128-bit load feeds the packed operations directly;
//  * squared distances are accumulated in coordinate order (first term a
//    rounded product, then one fused multiply-add per coordinate), the same
//    rounding sequence the FP32 selection is defined by;
//  * the library is visited in query order from the run nearest each warp's
//    queries (wrapping around); 16-point chunks whose bounding box lies
//    farther than every lane's threshold are skipped whole;
//  * selection: each query keeps the K = E+1 smallest distances seen as a
//    sorted float list in registers (a min/max network, no index
//    bookkeeping), which is its running threshold, and the (squared
//    distance, index) keys of every candidate at or below the threshold in
//    its column of a shared-memory buffer; the column is compacted when it
//    runs full and sorted at the end, so the E+1 nearest come out in
//    (distance, index) order however the library was visited;
//  * the epilogue forms u_i = exp(-d_i/d_1) (optionally floored), the
//    prediction, and the FP64 moments of each (tile, target): predictions go
//    to a shared-memory ring whose eight slots are reduced by eight warps at
//    once (the FP64 pipe is the scarce unit); the observed values' half is
//    done once per (j, i, E, tau) by obs_kernel, not once per realization;
//    the last (tile, target) of a realization to finish merges the tiles'
//    moments in a fixed order, so rho does not depend on the schedule.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <initializer_list>

#include "ccm_internal.h"

namespace ccm {
namespace {

using u64 = unsigned long long;

constexpr int kThreads = 256;             // threads per CTA = queries per tile
constexpr int kQT = kThreads;             // queries per tile (one per thread)
static_assert((kQT & (kQT - 1)) == 0, "tile moments rely on a power-of-two tile");
constexpr int kBuf = 20;                  // candidate keys per query (a column of the buffer)
constexpr int kCoordBytes = 24 * 1024;    // shared memory for one library tile + chunk boxes
constexpr int kBoxBytes = 4 * 1024;       // chunk bounding boxes, at the end of that region
constexpr int kChunk = 16;                // library points per bounding box
constexpr int kBufBytes = kBuf * kThreads * 8;
// Predictions staged for their FP64 moments: kRing (tile, target) vectors of
// kQT floats, reduced together, one warp each, when the ring is full.
constexpr int kRing = kThreads / 32;
constexpr int kRingBytes = kRing * kThreads * 4;
constexpr int kSmemBytes = kCoordBytes + kBufBytes + kRingBytes;
constexpr unsigned kFull = 0xffffffffu;
// Kernel variants picked per E by the autotuner (results are identical):
//   V = 0 "narrow": 4 library points per step, no early termination;
//   V = 1 "wide":   early termination for E >= 3 (after 2 coordinates for
//                   E <= 6, after 3 above), and 8 points per step for E <= 6
//                   (4 above: registers run out).

// Library points per step (two points per packed operand): more points give
// more independent FMA chains per warp.
template <int E, int V>
constexpr int kStepE = (V == 1 && E <= 6) ? 8 : 4;

// Coordinates summed before the early-termination check (E when there is none).
template <int E, int V>
constexpr int kE1 = (V == 1 && E >= 3) ? (E <= 6 ? 2 : 3) : E;

template <int E>
struct TileShape {
  static constexpr int EP = E + (E & 1);                        // coordinates padded to even
  static constexpr int D = E < 3 ? E : 3;                       // coordinates a chunk box bounds
  // library points per tile: a point pair takes EP*8 bytes of coordinates + 8 of indices
  static constexpr int LT = ((kCoordBytes - kBoxBytes) / (EP * 8 + 8)) * 2 / 64 * 64;
  static_assert(LT >= 64 && LT % 32 == 0, "tile must hold whole warps of chunks");
  static_assert((LT / kChunk) * 2 * D * 4 <= kBoxBytes, "chunk boxes must fit");
};

__device__ __forceinline__ u64 pack2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Squared distances of one query (coordinates duplicated, {q_e, q_e}) to a
// pair of library points whose coordinates are packed {a_e, b_e} starting at
// `c` (16-byte aligned, EP entries): {d2(q, a), d2(q, b)}, accumulated over
// coordinates [EB, EE) onto `acc` in the fixed order (coordinate 0 a rounded
// product, every later one a fused multiply-add).  Calling it for [0, E1)
// and then [E1, E) gives exactly the bits of one call for [0, E).
template <int E, int EB, int EE>
__device__ __forceinline__ u64 sqdist2_range(const u64 (&qc)[E], const u64* c, u64 acc) {
  const ulonglong2* c2 = reinterpret_cast<const ulonglong2*>(c);
#pragma unroll
  for (int e = EB & ~1; e < EE; e += 2) {
    const ulonglong2 v = c2[e / 2];
    if (e >= EB) {
      const u64 d0 = sub2(qc[e], v.x);
      acc = (e == 0) ? mul2(d0, d0) : fma2(d0, d0, acc);
    }
    if (e + 1 < EE && e + 1 >= EB) {
      const u64 d1 = sub2(qc[e + 1], v.y);
      acc = fma2(d1, d1, acc);
    }
  }
  return acc;
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Smallest of N distances (three-input min where possible).
template <int N>
__device__ __forceinline__ float min_all(const float (&d)[N]) {
  float m = d[0];
  int i = 1;
#pragma unroll
  for (; i + 1 < N; i += 2) m = min3f(m, d[i], d[i + 1]);
  if (i < N) m = fminf(m, d[i]);
  return m;
}

// The selection key: (squared distance, manifold index), lexicographic.
__device__ __forceinline__ bool key_less(float d, int l, float kd, int kl) {
  return d < kd || (d == kd && l < kl);
}

// The same key packed in 64 bits: the bits of a non-negative float order
// like its value, so (bits << 32 | index) compares like (d, index).
__device__ __forceinline__ u64 pack_key(float d, int l) {
  return ((u64)__float_as_uint(d) << 32) | (u64)(uint32_t)l;
}
__device__ __forceinline__ float key_dist(u64 k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int key_index(u64 k) { return (int)(uint32_t)k; }

// Insert key x into the ascending list ku[0..K); a no-op when x is not below
// the last entry.  The library is visited in any order.
template <int K>
__device__ __forceinline__ void insert_sorted(u64 (&ku)[K], u64 x) {
  bool below[K];
#pragma unroll
  for (int s = 0; s < K; ++s) below[s] = x < ku[s];
#pragma unroll
  for (int s = K - 1; s > 0; --s) ku[s] = below[s - 1] ? ku[s - 1] : (below[s] ? x : ku[s]);
  ku[0] = below[0] ? x : ku[0];
}

// Insert key x into ku[0..K) when only ku[0..n) may hold keys (the rest are
// the empty key): the same result as insert_sorted, with the comparisons of
// slots past n folded away when n is a compile-time constant.
template <int K>
__device__ __forceinline__ void insert_prefix(u64 (&ku)[K], u64 x, int n) {
  bool below[K];
#pragma unroll
  for (int s = 0; s < K; ++s) below[s] = (s <= n) && x < ku[s];
#pragma unroll
  for (int s = K - 1; s > 0; --s)
    if (s <= n) ku[s] = below[s - 1] ? ku[s - 1] : (below[s] ? x : ku[s]);
  ku[0] = below[0] ? x : ku[0];
}

// Butterfly sum over the warp: every lane ends with the same bits (each
// level adds the same two values in either order).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Two-pass FP64 moments of one tile's (observed x, predicted y) pairs, by one
// warp: each lane sums a fixed strided subset, then the butterfly.  The
// predictions are staged in shared memory (ys[0..nq)); the observed half comes
// from the tile's record (obs_kernel: x_q - mean(x), mean(x), Sxx), computed
// there with the same lane order and butterfly.  Writes (n, mean_x, mean_y,
// Sxx, Syy, Sxy) about the tile means.
constexpr int kPer = kQT / 32;  // queries per lane

// Mean of the nq lane-strided values v(c) = value lane + 32c (the sum in lane
// order, then the butterfly); a full tile divides by 256 = 2^8, and
// multiplying by 2^-8 gives the same bits and spares the FP64 pipe a division.
template <class V>
__device__ __forceinline__ double tile_mean(V v, int nq) {
  const int lane = threadIdx.x & 31;
  double sv = 0.0;
#pragma unroll
  for (int c = 0; c < kPer; ++c)
    if (lane + 32 * c < nq) sv = __dadd_rn(sv, v(c));
  sv = warp_sum(sv);
  return (nq == kQT) ? __dmul_rn(sv, 1.0 / kQT) : __ddiv_rn(sv, (double)nq);
}

__device__ __forceinline__ void tile_moments(const float* ys, const double* rec, int nq,
                                             double* part) {
  const int lane = threadIdx.x & 31;
  double y[kPer];
#pragma unroll
  for (int c = 0; c < kPer; ++c) y[c] = (double)ys[lane + 32 * c];
  const double my = tile_mean([&](int c) { return y[c]; }, nq);
  double syy = 0.0, sxy = 0.0;
#pragma unroll
  for (int c = 0; c < kPer; ++c) {
    const int q = lane + 32 * c;
    if (q < nq) {
      const double b = __dsub_rn(y[c], my);
      syy = __fma_rn(b, b, syy);
      sxy = __fma_rn(__ldg(rec + q), b, sxy);
    }
  }
  syy = warp_sum(syy);
  sxy = warp_sum(sxy);
  if (lane == 0) {
    part[0] = (double)nq;
    part[1] = __ldg(rec + kQT);
    part[2] = my;
    part[3] = __ldg(rec + kQT + 1);
    part[4] = syy;
    part[5] = sxy;
  }
}

// Observed-moment records (see ObsJob), one warp per tile: x_q is the target
// at the tile's manifold points (Sect. 2.1: the value the cross map
// predicts).  The same lane order and butterfly as tile_moments.
__global__ void __launch_bounds__(kThreads) obs_kernel(const float* series, const int32_t* order,
                                                      const ObsJob* jobs, int64_t n_jobs,
                                                      int64_t n_tiles, double* obs) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_tiles;
       g += n_warps) {
    int64_t lo = 0, hi = n_jobs - 1;  // the job holding tile g: last obs_tile <= g
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (jobs[mid].obs_tile <= g) lo = mid;
      else hi = mid - 1;
    }
    const ObsJob jb = jobs[lo];
    const int tile = (int)(g - jb.obs_tile);
    const int nq = min(kQT, jb.n_m - tile * kQT);
    const float* si = series + jb.series_off + (int64_t)jb.i * jb.n;
    const int32_t* ord = order + jb.order_off + (int64_t)tile * kQT;
    const int off = (jb.E - 1) * jb.tau;
    double x[kPer];
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
      const int q = lane + 32 * c;
      x[c] = (q < nq) ? (double)si[ord[q] + off] : 0.0;
    }
    const double mx = tile_mean([&](int c) { return x[c]; }, nq);
    double* rec = obs + g * kObsStride;
    double sxx = 0.0;
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
      const int q = lane + 32 * c;
      double a = 0.0;
      if (q < nq) {
        a = __dsub_rn(x[c], mx);
        sxx = __fma_rn(a, a, sxx);
      }
      rec[q] = a;
    }
    sxx = warp_sum(sxx);
    if (lane == 0) {
      rec[kQT] = mx;
      rec[kQT + 1] = sxx;
    }
  }
}

// Merge the tile moments of one (realization, target) into rho, by one warp.
// With the grand means MX = sum(n_t mx_t)/N, the centred sums are exactly
//   Sxx = sum_t [Sxx_t + n_t (mx_t - MX)^2]   (likewise Syy, Sxy),
// a sum of non-negative terms (no cancellation), taken in a fixed lane and
// butterfly order: rho does not depend on which CTA ran which tile, or when.
__device__ __forceinline__ double merge_moments(const double* base, int n_tiles) {
  const int lane = threadIdx.x & 31;
  double N = 0.0, SX = 0.0, SY = 0.0;
  for (int q = lane; q < n_tiles; q += 32) {
    const double* pt = base + 6 * q;
    const double nq = __ldcg(pt + 0);
    N = __dadd_rn(N, nq);
    SX = __fma_rn(nq, __ldcg(pt + 1), SX);
    SY = __fma_rn(nq, __ldcg(pt + 2), SY);
  }
  N = warp_sum(N);
  SX = warp_sum(SX);
  SY = warp_sum(SY);
  const double MX = __ddiv_rn(SX, N), MY = __ddiv_rn(SY, N);
  double SXX = 0.0, SYY = 0.0, SXY = 0.0;
  for (int q = lane; q < n_tiles; q += 32) {
    const double* pt = base + 6 * q;
    const double nq = __ldcg(pt + 0);
    const double dx = __dsub_rn(__ldcg(pt + 1), MX), dy = __dsub_rn(__ldcg(pt + 2), MY);
    const double wx = __dmul_rn(nq, dx);
    SXX = __fma_rn(wx, dx, __dadd_rn(SXX, __ldcg(pt + 3)));
    SYY = __fma_rn(__dmul_rn(nq, dy), dy, __dadd_rn(SYY, __ldcg(pt + 4)));
    SXY = __fma_rn(wx, dy, __dadd_rn(SXY, __ldcg(pt + 5)));
  }
  SXX = warp_sum(SXX);
  SYY = warp_sum(SYY);
  SXY = warp_sum(SXY);
  return (SXX > 0.0 && SYY > 0.0) ? __ddiv_rn(SXY, __dsqrt_rn(__dmul_rn(SXX, SYY))) : nan("");
}

// Called by a reducer warp after its lane 0 wrote the moments of one (tile,
// target) of a realization: the fence orders them before the completion
// count, and the last of the realization's n_tiles * n_targets to arrive
// merges every target's moments.  Out of line: inlined its registers would
// crowd the search.
__device__ __noinline__ void complete_tile(const KnnParams& p, int unit) {
  const int lane = threadIdx.x & 31;
  unsigned prev = 0u;
  if (lane == 0) {
    __threadfence();
    prev = atomicAdd(&p.unit_done[unit], 1u);
  }
  prev = __shfl_sync(kFull, prev, 0);
  const UnitDesc& u = p.units[unit];
  const int n_tiles = u.n_tiles, n_targets = u.n_targets;
  if (prev != (unsigned)(n_tiles * n_targets - 1)) return;
  __threadfence();
  for (int t = 0; t < n_targets; ++t) {
    const double r = merge_moments(p.partials + 6 * (u.part_off + (int64_t)t * n_tiles), n_tiles);
    if (lane == 0) p.rho[p.targets[u.tgt_off + t].out_idx] = r;
  }
  if (lane == 0) p.unit_done[unit] = 0u;  // ready for the next run
}

// A staged (tile, target) prediction vector awaiting its FP64 moments.
struct RingMeta {
  const double* rec;  // the tile's observed-value record
  double* part;       // where its six moments go
  int32_t unit;       // its realization
  int32_t nq;         // valid queries of the tile
};

// The staged vectors' moments: warps 0..n-1 take one each, in parallel (so the
// FP64 pipes of all four SM sub-partitions share the work), and count it
// towards its realization's completion.  Between two block barriers: the
// slots are complete on entry and free again on exit.
__device__ __forceinline__ void flush_ring(const KnnParams& p, const float* ring,
                                           const RingMeta* meta, int n) {
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  if (warp < n) {
    const RingMeta mt = meta[warp];
    tile_moments(ring + warp * kQT, mt.rec, mt.nq, mt.part);
    complete_tile(p, mt.unit);
  }
  __syncthreads();
}

// Everything after the neighbour search, shared by the brute-force and the
// table paths: dd[0..E] ascending FP32 squared distances (kDist: their
// distances sqrt_hw(d2) already) and nb[0..E] the neighbours of query m
// (itself excluded).  Simplex weights and the
// prediction of every target; each target's prediction vector goes to the
// next ring slot (ring_n, the same in every thread), and a full ring is
// reduced (flush_ring).  The CTA flushes what is left when it runs out of
// work.  rho does not depend on which warp reduced which vector, or when.
// `keep` (brute-force path: the thread's own column of the candidate buffer,
// which only this thread uses and which is free once its search is done)
// holds the weights and neighbours in shared memory, so that a reduction
// between two targets finds no live registers to spill; other warps may still
// be searching, so nothing else of the buffer is touched.  kKeep false: they
// stay in registers.  nb_values (table path, one target, no checking copy of
// the neighbours): nb holds the bits of the target's values at the E+1
// neighbours, read from the table instead of gathered.
static_assert(kMaxE + 1 <= kBuf, "the epilogue keeps E+1 entries in a candidate column");
template <int E, bool kKeep, bool kDist = false>
__device__ __forceinline__ void finish_tile(const KnnParams& p, const UnitDesc& u, int unit,
                                            int tile, int m, bool valid, const float (&dd)[E + 1],
                                            const int (&nb)[E + 1], float* ring, RingMeta* meta,
                                            int& ring_n, u64* keep, bool nb_values = false) {
  const int tid = threadIdx.x;
  const int n_m = u.n_m;
  const int off = (E - 1) * u.tau;
  const int nq = min(kQT, n_m - tile * kQT);  // valid queries of this tile (>= 1)
  // Simplex weights (Sect. 2.1), once per query for every target.  Every
  // floating-point step below is a fixed operation (explicit rounding or a
  // hardware approximation that is the same everywhere), so the brute-force
  // and table kernels, the plain comparator and every batch produce the same
  // bits.
  const float d1 = kDist ? dd[0] : sqrt_hw(dd[0]);
  const float inv_d1 = (d1 > 0.f) ? rcp_hw(d1) : 0.f;
  float w[E + 1];
  int nbc[E + 1];
  float usum = 0.f;
  // simplex_u_dist with the d1 > 0 test taken once: the exponential for every
  // neighbour, replaced by the limit in the rare query whose nearest is at 0
#pragma unroll
  for (int s = 0; s <= E; ++s) w[s] = simplex_exp(kDist ? dd[s] : sqrt_hw(dd[s]), inv_d1);
  if (!(d1 > 0.f)) {
#pragma unroll
    for (int s = 0; s <= E; ++s) w[s] = simplex_limit(kDist ? dd[s] : sqrt_hw(dd[s]));
  }
#pragma unroll
  for (int s = 0; s <= E; ++s) {
    w[s] = fmaxf(w[s], u.wfloor);
    usum = __fadd_rn(usum, w[s]);
    // brute force: an unfilled slot (only possible with non-finite device
    // input) reads, and is reported, in bounds; table entries are in bounds
    nbc[s] = kDist ? nb[s] : min(max(nb[s], 0), n_m - 1);
    if (kKeep) keep[s * kThreads + tid] = ((u64)__float_as_uint(w[s]) << 32) | (uint32_t)nbc[s];
  }
  auto weight = [&](int s) {
    return kKeep ? __uint_as_float((uint32_t)(keep[s * kThreads + tid] >> 32)) : w[s];
  };
  auto nbr = [&](int s) { return kKeep ? (int)(uint32_t)keep[s * kThreads + tid] : nbc[s]; };
  for (int t = 0; t < u.n_targets; ++t) {
    const TargetDesc tg = p.targets[u.tgt_off + t];
    const float* si = p.series + u.series_off + (int64_t)tg.i * u.n;
    float acc = 0.f;
    if (nb_values) {  // nb holds the table's copy of the target at the neighbours
#pragma unroll
      for (int s = 0; s <= E; ++s) acc = __fmaf_rn(weight(s), __int_as_float(nbr(s)), acc);
    } else {
#pragma unroll
      for (int s = 0; s <= E; ++s) acc = __fmaf_rn(weight(s), si[nbr(s) + off], acc);
    }
    const float xhat = __fmul_rn(acc, rcp_hw(usum));  // usum >= exp(-1)
    if (valid) {
      if (p.dbg_xhat) p.dbg_xhat[tg.q_off + m] = xhat;
      if (p.dbg_nbr) {
#pragma unroll
        for (int s = 0; s <= E; ++s) p.dbg_nbr[tg.nbr_off + (int64_t)m * (E + 1) + s] = nbr(s);
      }
    }
    ring[ring_n * kQT + tid] = valid ? xhat : 0.f;
    if (tid == 0)
      meta[ring_n] = RingMeta{p.obs + (tg.obs_tile + tile) * kObsStride,
                              p.partials + 6 * (u.part_off + (int64_t)t * u.n_tiles + tile), unit,
                              nq};
    // a full ring is reduced before the next target's vector, or at the end
    if (++ring_n == kRing && t + 1 < u.n_targets) {
      flush_ring(p, ring, meta, kRing);
      ring_n = 0;
    }
  }
  if (ring_n == kRing) {  // the weights and neighbours are dead here
    flush_ring(p, ring, meta, kRing);
    ring_n = 0;
  }
}

// Stage library points [t0, t0 + nt) of a unit's library (query order) into
// shared memory: coordinates in packed pairs, indices, and the bounding box
// of every kChunk consecutive points over the first D coordinates.  The tile
// is padded to whole chunks with sentinel points (NaN coordinates, index
// INT_MAX) that are never selected.  Block-wide; the caller brackets it with
// barriers.  Sentinel coordinates are NaN: every distance to a sentinel is
// NaN, which compares false against any threshold.
template <int E>
__device__ __noinline__ void stage_library(const float* sj, const int32_t* lib, int off, int tau,
                                              int t0, int nt, u64* s_coord, int32_t* s_lidx,
                                              float* s_box) {
  constexpr int EP = TileShape<E>::EP;
  constexpr int D = TileShape<E>::D;
  const int tid = threadIdx.x;
  const int ntp = (nt + kChunk - 1) / kChunk * kChunk;
  for (int a = tid; a < (ntp + 31) / 32 * 32; a += kThreads) {  // whole warps: the box shuffles
    const int pp = a >> 1, half = a & 1;
    float c0[D];
    if (a < nt) {
      const int l = lib[t0 + a];
      s_lidx[a] = l;
      float* cpair = reinterpret_cast<float*>(s_coord + (size_t)pp * EP);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const float c = sj[l + off - e * tau];
        cpair[2 * e + half] = c;
        if (e < D) c0[e] = c;
      }
      if (EP > E) cpair[2 * E + half] = 0.f;
    } else {
      if (a < ntp) {  // sentinel point: never selected
        s_lidx[a] = INT_MAX;
        float* cpair = reinterpret_cast<float*>(s_coord + (size_t)pp * EP);
#pragma unroll
        for (int e = 0; e < E; ++e) cpair[2 * e + half] = __int_as_float(0x7fffffff);
        if (EP > E) cpair[2 * E + half] = 0.f;
      }
#pragma unroll
      for (int e = 0; e < D; ++e) c0[e] = __int_as_float(0x7fffffff);
    }
    // chunk boxes over the first D coordinates: one per half-warp (fminf and
    // fmaxf skip the NaN of a sentinel; a chunk always holds a real point)
#pragma unroll
    for (int e = 0; e < D; ++e) {
      float lo = c0[e], hi = c0[e];
#pragma unroll
      for (int o = kChunk / 2; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
      }
      if ((a & (kChunk - 1)) == 0 && a < ntp) {
        s_box[(a / kChunk) * 2 * D + e] = lo;
        s_box[(a / kChunk) * 2 * D + D + e] = hi;
      }
    }
  }
}

// The library position (in query order) about as far into the library as
// query position pos is into the manifold: floor(L*pos/N_m), in FP32 (only a
// starting point of the scan: any value in [0, L) gives the same result).
__device__ __forceinline__ int library_position(int L, int pos, int n_m) {
  return min(L - 1, __float2int_rz(__fmul_rn((float)L, __fdividef((float)pos, (float)n_m))));
}

// The running threshold: t[0..K) holds the K smallest squared distances (as
// values, ties repeated) of the candidates seen so far, ascending.  Inserting
// x is a min/max network: slot s becomes min(t[s], max(t[s-1], x)), which
// leaves the list unchanged when x is not below t[K-1].
template <int K>
__device__ __forceinline__ void thresh_insert(float (&t)[K], float x) {
#pragma unroll
  for (int s = K - 1; s > 0; --s) t[s] = fminf(t[s], fmaxf(t[s - 1], x));
  t[0] = fminf(t[0], x);
}

// Ascending insertion sort of one thread's candidate column (n keys, stride
// kThreads) in shared memory.
__device__ __forceinline__ void sort_column(u64* col, int n) {
  for (int i = 1; i < n; ++i) {
    const u64 x = col[i * kThreads];
    int j = i - 1;
    for (; j >= 0; --j) {
      const u64 y = col[j * kThreads];
      if (y <= x) break;
      col[(j + 1) * kThreads] = y;
    }
    col[(j + 1) * kThreads] = x;
  }
}

// Brute-force search of one work item: query tiles [tile0, tile0 +
// kBruteChunk) of a unit.  When the whole library fits one shared-memory tile
// it is staged once for all of them; each warp starts its scan at the library
// run nearest its own 32 queries (the library is in query order) and wraps
// around.  Larger libraries are staged tile by tile for every query tile.
//
// Selection.  Each query keeps (a) the running threshold t[] of the K = E+1
// smallest squared distances seen (registers, min/max network) and (b) a
// column of the candidate buffer in shared memory with the keys (squared
// distance, index) of every candidate whose distance was at most the threshold
// when it was seen.  Every key that can still be among the final K smallest
// is in the column: a dropped key had a distance above a threshold that is
// itself at least the final K-th smallest value.  The threshold is brought up
// to date warp-wide once some lane has merge_at new candidates (the network is
// cheap: no index bookkeeping); a nearly full column is compacted to the keys
// at or below the threshold, and, if ties still leave it full, sorted and cut
// to the K smallest keys.  At the end the column is compacted and sorted: its
// first K keys are the E+1 nearest neighbours in (distance, index) order,
// exactly the list the sorted insertion of every candidate would give.
template <int E, int V, bool kStats>
__device__ void process_item(const KnnParams& p, const UnitDesc& u, int unit, int tile0,
                             unsigned char* smem, RingMeta* meta, int& ring_n) {
  constexpr int K = E + 1;  // the window keeps m itself out, so E+1 slots suffice
  constexpr int EP = TileShape<E>::EP;
  constexpr int LT = TileShape<E>::LT;
  constexpr int D = TileShape<E>::D;
  const int n_m = u.n_m, L = u.L, tau = u.tau, W = u.theiler;
  const bool single = L <= LT;
  // Shared-memory layout: library indices [LT], chunk boxes [LT/kChunk][2D],
  // coordinates [LT/2][EP] in the first kCoordBytes, then the candidate
  // buffer [kBuf][kThreads].  A library that fits one tile takes only the
  // coordinate rows it needs, and the buffer starts right after them, so its
  // columns reach up to the prediction ring: wider columns need fewer
  // compactions.
  int32_t* s_lidx = reinterpret_cast<int32_t*>(smem);
  float* s_box = reinterpret_cast<float*>(smem + (size_t)LT * 4);
  u64* s_coord = reinterpret_cast<u64*>(smem + (size_t)LT * 4 + kBoxBytes);
  size_t buf_off = kCoordBytes;
  if (single) {
    const int ntp = (L + kChunk - 1) / kChunk * kChunk;
    buf_off = (size_t)LT * 4 + kBoxBytes + (size_t)(ntp / 2) * EP * 8;
  }
  u64* s_buf = reinterpret_cast<u64*>(smem + buf_off);
  const int cap = (int)((kCoordBytes + kBufBytes - buf_off) / (kThreads * 8));  // >= kBuf
  float* s_ring = reinterpret_cast<float*>(smem + kCoordBytes + kBufBytes);      // [kRing][kQT]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int off = (E - 1) * tau;
  const float* sj = p.series + u.series_off + (int64_t)u.j * u.n;
  const int32_t* lib = p.lib + u.lib_off;
  const int32_t* order = p.order + u.order_off;
  constexpr int kStep = kStepE<E, V>;
  constexpr int kPairs = kStep / 2;
  const int room = cap - kStep;   // a column above this cannot take another step
  static_assert(K + kStep <= kBuf, "a cut column must leave room for a step");
  const int merge_at = max(1, min(p.merge_at[E], room));
  // the first kInit points of a query's scan go straight into its threshold
  constexpr int kInit = (K + kStep - 1) / kStep * kStep;
  static_assert(kInit <= kChunk, "the initial points lie in the first chunk");
  u64* col = s_buf + tid;  // this thread's candidate column

  const int tile1 = min(u.n_tiles, tile0 + kBruteChunk);
  if (single) {
    __syncthreads();  // the previous item's readers of the tile are done
    stage_library<E>(sj, lib, off, tau, 0, L, s_coord, s_lidx, s_box);
    __syncthreads();
  }
  // A warp's 32 queries are consecutive positions of the query order.  For
  // small E (a short search, so the load latency would show) the next tile's
  // query and coordinates are loaded before this tile's epilogue, so their
  // latency overlaps it; for larger E the registers are needed elsewhere.
  constexpr bool kPrefetch = E <= 3;
  int m_nx;
  float c_nx[E];
  auto load_query = [&](int t) {
    const int ps = t * kQT + tid;
    m_nx = order[ps < n_m ? ps : n_m - 1];
#pragma unroll
    for (int e = 0; e < E; ++e) c_nx[e] = sj[m_nx + off - e * tau];
  };
  if (kPrefetch) load_query(tile0);
  for (int tile = tile0; tile < tile1; ++tile) {
    if (!kPrefetch) load_query(tile);
    const int pos = tile * kQT + tid;
    const bool valid = pos < n_m;
    const int m = m_nx;
    u64 qc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) qc[e] = pack2(c_nx[e], c_nx[e]);
    // Bounding box of the warp's queries over the first D coordinates.
    float qlo[D], qhi[D];
#pragma unroll
    for (int e = 0; e < D; ++e) {
      float lo = c_nx[e], hi = lo;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
      }
      qlo[e] = lo;
      qhi[e] = hi;
    }
    // the library position nearest this warp's queries (in query order)
    const int aw = library_position(L, tile * kQT + warp * 32, n_m);

    float tl[K];  // running threshold: the K smallest distances so far, ascending
#pragma unroll
    for (int s = 0; s < K; ++s) tl[s] = INFINITY;
    int cnt = 0, done = 0;  // keys in the column; of them, already in tl
    // counting variant only: warp-uniform step counts, per-lane candidates
    uint32_t st_begun = 0, st_full = 0, st_pruned = 0, st_cand = 0, st_slots = 0;

    // bring tl up to date with the column's new keys (lockstep over the lanes)
    auto update = [&]() {
      const int mx = (int)__reduce_max_sync(kFull, (unsigned)(cnt - done));
      if (kStats) {
        st_cand += (uint32_t)(cnt - done);
        st_slots += (uint32_t)mx;
      }
      for (int b = 0; b < mx; ++b) {
        // the distance half of the key; a lane with no new key inserts +inf
        // (a no-op), and a round no lane needs any more is skipped
        const float x = (b < cnt - done)
                            ? reinterpret_cast<const float*>(col + (done + b) * kThreads)[1]
                            : INFINITY;
        if (__any_sync(kFull, x < tl[K - 1])) thresh_insert<K>(tl, x);
      }
      done = cnt;
    };
    // keep the keys at or below the threshold (in order)
    auto compact = [&]() {
      const float th = tl[K - 1];
      const int mx = (int)__reduce_max_sync(kFull, (unsigned)cnt);
      int w = 0;
      for (int b = 0; b < mx; ++b) {
        if (b < cnt) {
          const u64 x = col[b * kThreads];
          if (key_dist(x) <= th) col[(w++) * kThreads] = x;
        }
      }
      cnt = done = w;
    };
    auto make_room = [&]() {
      update();
      if (__any_sync(kFull, cnt > room)) compact();
      if (__any_sync(kFull, cnt > room)) {  // ties at the threshold: keep the K smallest keys
        if (cnt > room) {
          sort_column(col, cnt);
          cnt = done = K;
        }
      }
    };

    // Scan the staged points [0, nt) from position `base` (a chunk start),
    // wrapping around; `first`: the scan's first kInit points fill tl.
    // Scan the staged points [0, nt) chunk by chunk from the chunk at `base`,
    // wrapping around; `first`: the scan's first kInit points fill tl.
    auto scan = [&](int nt, int base, bool first) {
      const int ntp = (nt + kChunk - 1) / kChunk * kChunk;
      const int nch = ntp / kChunk;
      const int c0 = base / kChunk;
      constexpr int kSteps = kChunk / kStep;  // steps per chunk
      if (first) {
#pragma unroll
        for (int pp = 0; pp < kInit / 2; ++pp) {
          const int a = base + 2 * pp;
          float d2[2];
          unpack2(sqdist2_range<E, 0, E>(qc, s_coord + (size_t)(a >> 1) * EP, 0ull), d2[0], d2[1]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int l = s_lidx[a + h];
            if (l != INT_MAX && abs(l - m) > W) {
              thresh_insert<K>(tl, d2[h]);
              col[(cnt++) * kThreads] = pack_key(d2[h], l);
            }
          }
        }
        done = cnt;
        if (kStats) {
          st_begun += kInit;
          st_full += kInit;
        }
        if (__any_sync(kFull, cnt > room)) make_room();
      }
#pragma unroll 1
      for (int jc = 0; jc < nch; ++jc) {
        int c = c0 + jc;
        c -= (c >= nch) ? nch : 0;
        const int s0 = (first && jc == 0) ? kInit / kStep : 0;  // steps the fill took
        if (s0 == 0) {
          // Chunk pruning.  gap_e = max(0, lo_e - qhi_e, qlo_e - hi_e) bounds
          // |q_e - x_e| from below for every query q of the warp and point x of
          // the chunk, in FP32 too (rounding is monotone); summed in the
          // distance's own order over the first D coordinates it bounds every
          // FP32 squared distance between them from below.  A chunk whose bound
          // exceeds every lane's threshold holds no candidate.
          const float* bx = s_box + c * 2 * D;
          float lb = 0.f;
#pragma unroll
          for (int e = 0; e < D; ++e) {
            const float g = fmaxf(fmaxf(__fsub_rn(bx[e], qhi[e]), __fsub_rn(qlo[e], bx[D + e])), 0.f);
            lb = (e == 0) ? __fmul_rn(g, g) : __fmaf_rn(g, g, lb);
          }
          const float th_max = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(tl[K - 1])));
          if (lb > th_max) {
            if (kStats) st_pruned += kChunk;
            continue;
          }
        }
        // two steps a chunk (kStep 8) unrolled; four (kStep 4, the larger E)
        // kept as a loop: unrolled they outgrow the instruction cache
#pragma unroll(kSteps <= 2 ? kSteps : 1)
        for (int sp = s0; sp < kSteps; ++sp) {
          const int a = c * kChunk + sp * kStep;
          if (kStats) st_begun += kStep;
          const u64* cp = s_coord + (size_t)(a >> 1) * EP;
          // Partial sums over the first E1 coordinates are lower bounds of the
          // full FP32 sums (all terms are >= 0 and rounding is monotone), so a
          // step whose partials are all above every lane's threshold cannot
          // contribute a candidate and skips the remaining coordinates.
          u64 r[kPairs];
#pragma unroll
          for (int pp = 0; pp < kPairs; ++pp) r[pp] = sqdist2_range<E, 0, (kE1<E, V>)>(qc, cp + pp * EP, 0ull);
          const float th = tl[K - 1];
          float d[kStep];
#pragma unroll
          for (int pp = 0; pp < kPairs; ++pp) unpack2(r[pp], d[2 * pp], d[2 * pp + 1]);
          if (kStats && (kE1<E, V>) == E) st_full += kStep;
          if (!__any_sync(kFull, min_all(d) <= th)) continue;
          if constexpr ((kE1<E, V>) < E) {
            if (kStats) st_full += kStep;
#pragma unroll
            for (int pp = 0; pp < kPairs; ++pp) {
              r[pp] = sqdist2_range<E, (kE1<E, V>), E>(qc, cp + pp * EP, r[pp]);
              unpack2(r[pp], d[2 * pp], d[2 * pp + 1]);
            }
            if (!__any_sync(kFull, min_all(d) <= th)) continue;
          }
          // the step's library indices (one broadcast 16-byte load per four)
          int li[kStep];
#pragma unroll
          for (int q4 = 0; q4 < kStep / 4; ++q4) {
            const int4 v = *reinterpret_cast<const int4*>(s_lidx + a + 4 * q4);
            li[4 * q4] = v.x;
            li[4 * q4 + 1] = v.y;
            li[4 * q4 + 2] = v.z;
            li[4 * q4 + 3] = v.w;
          }
#pragma unroll
          for (int pt = 0; pt < kStep; ++pt) {
            // at or below the threshold (never a sentinel: NaN), outside the
            // exclusion window |l - m| <= W (W = 0 drops only m itself, and
            // the unsigned form tests both sides at once); appended without a
            // branch
            const bool take = (d[pt] <= th) &
                              ((unsigned)li[pt] - (unsigned)m + (unsigned)W > 2u * (unsigned)W);
            if (take) col[cnt * kThreads] = pack_key(d[pt], li[pt]);
            cnt += take ? 1 : 0;
          }
          if (__any_sync(kFull, cnt - done >= merge_at || cnt > room)) make_room();
        }
      }
    };

    // The library is staged tile by tile unless it fits one shared-memory tile
    // (staged once per item above); the first library tile visited is the one
    // nearest this query tile (the same order in every warp: the staging is
    // block-wide).
    const int ntiles = single ? 1 : (L + LT - 1) / LT;
    const int first_t = single ? 0 : library_position(L, tile * kQT, n_m) / LT;
    for (int c = 0; c < ntiles; ++c) {
      int ti = first_t + c;
      ti -= (ti >= ntiles) ? ntiles : 0;
      const int t0 = ti * LT, nt = min(LT, L - t0);
      if (!single) {
        __syncthreads();  // the previous library tile has been consumed
        stage_library<E>(sj, lib, off, tau, t0, nt, s_coord, s_lidx, s_box);
        __syncthreads();
      }
      const int local = aw - t0;
      const int base = (local >= 0 && local < nt) ? (local / kChunk) * kChunk : 0;
      scan(nt, base, c == 0);
    }
    update();
    compact();
    sort_column(col, cnt);  // the first K keys: the E+1 nearest, in (distance, index) order
    if (kStats) {
      const uint32_t cand = __reduce_add_sync(kFull, st_cand);
      const unsigned vq = __popc(__ballot_sync(kFull, valid));
      if (lane == 0) {
        unsigned long long* c = p.stats;
        atomicAdd(&c[kStatPairsBegun], 32ull * st_begun);
        atomicAdd(&c[kStatPairsFull], 32ull * st_full);
        atomicAdd(&c[kStatPairsPruned], 32ull * st_pruned);
        atomicAdd(&c[kStatCandidates], (unsigned long long)cand);
        atomicAdd(&c[kStatMergeSlots], 32ull * st_slots);
        atomicAdd(&c[kStatBruteQueries], (unsigned long long)vq);
        if (tid == 0) atomicAdd(&c[kStatBruteTiles], 1ull);
      }
    }

    // Epilogue: the E+1 nearest (the window kept the query itself out of the
    // list), simplex weights, prediction, moments.
    float dd[E + 1];
    int nb[E + 1];
#pragma unroll
    for (int s = 0; s <= E; ++s) {
      const u64 k = col[s * kThreads];
      dd[s] = key_dist(k);
      nb[s] = key_index(k);
    }
    if (kPrefetch && tile + 1 < tile1) load_query(tile + 1);
    finish_tile<E, true>(p, u, unit, tile, m, valid, dd, nb, s_ring, meta, ring_n, s_buf);
    // the next tile's search starts behind a barrier (this also keeps the
    // search's registers free of spills)
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Table path: the library's members are marked in a shared-memory bitmap and
// each query walks its row of the distance indexing table (sorted by (FP32
// squared distance, index) over the whole manifold, the query itself left
// out) until it has met E+1 library members outside the exclusion window.  Those are, in order, the E+1 nearest
// library neighbours -- the same list the brute-force scan produces.  A query
// whose R table entries hold fewer members falls back to scanning the library.
template <int E>
__device__ __forceinline__ float d2_point(const float* sj, int off, int tau, const float (&q)[E],
                                          int x) {
  float diff = __fsub_rn(q[0], sj[x + off]);
  float acc = __fmul_rn(diff, diff);
#pragma unroll
  for (int e = 1; e < E; ++e) {
    diff = __fsub_rn(q[e], sj[x + off - e * tau]);
    acc = __fmaf_rn(diff, diff, acc);
  }
  return acc;
}

// Shared memory of the table kernel: the epilogue's ring of predictions, the
// walk's records (below), then the library membership map: one byte per
// manifold point when the manifold has at most kByteMapMax points (bit b: the
// point is in realization b's library), else one bit (one realization).
//
// A record is one step of the walk (eight consecutive ranks of the row) that
// held members of a realization: (step << 8) | flags, flag c marking rank
// 8*step + c.  A realization stops recording once it has E+1 members, so it
// keeps at most E+1 records: [kTableGroup][kMaxE+1][kThreads] 16-bit words.
constexpr int kRecBytes = kTableGroup * (kMaxE + 1) * kThreads * 2;
constexpr int kByteMapMax = 32768;
static_assert(kTableMaxR / 8 <= 256, "a record's step index has eight bits");
static_assert(kTableGroupMaxNm <= kByteMapMax, "grouped table items need the byte map");
static_assert(kTableGroup <= 4, "one byte of member flags per realization in 32 bits");

// One query's walk along its table row (see process_table_item): `at` is the
// element of its rank group 0, `rec` its column of the records, and act,
// counts and nrec the per-realization bytes described there.  The map is a
// byte map (kBytes) or a bitmap, fixed per work item, so each kind gets its
// own loop.
template <int K, bool kBytes, bool kStats>
__device__ __forceinline__ void table_walk(const KnnParams& p, int64_t at, int n_m, int groups, int m,
                                           int W, const unsigned char* map, uint16_t* rec,
                                           uint32_t& act, uint32_t& counts, uint32_t& nrec,
                                           uint32_t& st_entries) {
  const uint32_t table_limit = (uint32_t)(0x80 - K) * 0x01010101u;
  for (int g = 0; __any_sync(kFull, act != 0u && g < groups); g += 2) {
    const bool w0 = act != 0u && g < groups, w1 = act != 0u && g + 1 < groups;
    if (kStats) st_entries += (w0 ? 4u : 0u) + (w1 ? 4u : 0u);
    int x[8];  // ranks 4g .. 4g+7 of this query's row (index 0 when not loaded)
    if (p.table_u16) {
      const uint16_t* t16 = static_cast<const uint16_t*>(p.table) + at;
      const uint2 v0 = w0 ? __ldg(reinterpret_cast<const uint2*>(t16 + (int64_t)g * 4 * n_m))
                          : make_uint2(0u, 0u);
      const uint2 v1 = w1 ? __ldg(reinterpret_cast<const uint2*>(t16 + (int64_t)(g + 1) * 4 * n_m))
                          : make_uint2(0u, 0u);
      x[0] = v0.x & 0xffffu; x[1] = v0.x >> 16; x[2] = v0.y & 0xffffu; x[3] = v0.y >> 16;
      x[4] = v1.x & 0xffffu; x[5] = v1.x >> 16; x[6] = v1.y & 0xffffu; x[7] = v1.y >> 16;
    } else {
      const int32_t* t32 = static_cast<const int32_t*>(p.table) + at;
      const int4 v0 = w0 ? __ldg(reinterpret_cast<const int4*>(t32 + (int64_t)g * 4 * n_m))
                         : make_int4(0, 0, 0, 0);
      const int4 v1 = w1 ? __ldg(reinterpret_cast<const int4*>(t32 + (int64_t)(g + 1) * 4 * n_m))
                         : make_int4(0, 0, 0, 0);
      x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
      x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
    }
    // member flags: the map byte's bit b moved to bit c of byte b (the
    // multiply spreads bits 0..3 to bits 0, 8, 16, 24)
    uint32_t flags = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint32_t mb = kBytes ? (uint32_t)map[x[c]]
                                 : ((reinterpret_cast<const uint32_t*>(map)[x[c] >> 5] >> (x[c] & 31)) & 1u);
      flags |= (kBytes ? ((mb * 0x00204081u) & 0x01010101u) : mb) << c;  // a bitmap: one realization
    }
    flags &= act & ((w0 ? 0x0f0f0f0fu : 0u) | (w1 ? 0xf0f0f0f0u : 0u));
    if (W > 0) {
      // points inside the exclusion window |x - m| <= W are no neighbours
      // (the row never holds m itself, so W = 0 excludes nothing)
      uint32_t win = 0u;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        win |= (((unsigned)x[c] - (unsigned)m + (unsigned)W <= 2u * (unsigned)W) ? 1u : 0u) << c;
      flags &= ~(win * 0x01010101u);
    }
    if (flags != 0u) {
      // one record per realization with members in this step
#pragma unroll
      for (int b = 0; b < kTableGroup; ++b) {
        const uint32_t fb = (flags >> (8 * b)) & 0xffu;
        if (fb != 0u) {
          const uint32_t i = (nrec >> (8 * b)) & 0xffu;  // < K: the realization was short
          rec[(b * K + (int)i) * kThreads] = (uint16_t)(((uint32_t)(g >> 1) << 8) | fb);
          nrec += 1u << (8 * b);
        }
      }
      // per-byte population counts, then the realizations now complete
      uint32_t v = flags - ((flags >> 1) & 0x55555555u);
      v = (v & 0x33333333u) + ((v >> 2) & 0x33333333u);
      counts += (v + (v >> 4)) & 0x0f0f0f0fu;  // each byte stays below K + 8
      const uint32_t done = ((counts + table_limit) & 0x80808080u) >> 7;  // counts_b >= K
      act &= ~(done * 0xffu);
    }
  }
}

template <int E, bool kStats>
__device__ void process_table_item(const KnnParams& p, int unit0, int count, int tile0,
                                   unsigned char* smem, RingMeta* meta, int& ring_n) {
  // `count` consecutive realizations of one cell (the same manifold, table, L
  // and target; count > 1 only with a byte map): one walk of each query's row
  // finds the E+1 nearest members of every one of them.
  constexpr int K = E + 1;
  const int tid = threadIdx.x;
  const UnitDesc u0 = p.units[unit0];
  const int n_m = u0.n_m, L = u0.L, tau = u0.tau, R = u0.table_R, W = u0.theiler;
  const int off = (E - 1) * tau;
  const float* sj = p.series + u0.series_off + (int64_t)u0.j * u0.n;
  float* s_ring = reinterpret_cast<float*>(smem);
  uint16_t* s_rec = reinterpret_cast<uint16_t*>(smem + kRingBytes);  // [count][K][kThreads]
  unsigned char* map = smem + kRingBytes + kRecBytes;
  const bool bytes = n_m <= kByteMapMax;
  const int words = bytes ? (n_m + 3) >> 2 : (n_m + 31) >> 5;  // 32-bit words of the map
  uint32_t* mw = reinterpret_cast<uint32_t*>(map);
  // Library membership, once for the item's tiles: byte x holds bit b when
  // point x is in realization b's library (a bitmap of one realization for
  // manifolds above kByteMapMax points).
  __syncthreads();  // the previous item's readers of the map are done
  for (int w = tid; w < words; w += kThreads) mw[w] = 0u;
  __syncthreads();
  for (int b = 0; b < count; ++b) {
    const int32_t* lib = p.lib + p.units[unit0 + b].lib_off;
    for (int a = tid; a < L; a += kThreads) {
      const int l = lib[a];
      if (!bytes) atomicOr(&mw[l >> 5], 1u << (l & 31));
      else if (count == 1) map[l] = 1;
      else atomicOr(&mw[l >> 2], (1u << b) << (8 * (l & 3)));
    }
  }
  __syncthreads();

  const int tile1 = min(u0.n_tiles, tile0 + kTableChunk);
  const int groups = R >> 2;  // groups of four ranks
  const uint32_t all = (count >= 4) ? 0xffffffffu : (1u << (8 * count)) - 1u;
  for (int tile = tile0; tile < tile1; ++tile) {
    const int pos = tile * kQT + tid;
    const bool valid = pos < n_m;
    const int m = p.order[u0.order_off + (valid ? pos : n_m - 1)];

    // Walk the row (every manifold point but m, in (distance, index) order),
    // eight ranks a step; for each realization the first E+1 members outside
    // the window are its neighbours, in order.  Everything below works on four bytes at once,
    // byte b for realization b: `flags` the step's members (bit c: rank
    // 8*step + c), `counts` the members found so far, `act` 0xff while a
    // realization still lacks some, `nrec` its records.
    uint32_t act = valid ? all : 0u, counts = 0u, nrec = 0u;
    const int64_t col = (int64_t)(valid ? pos : 0) * 4;
    uint32_t st_entries = 0;
    if (bytes)
      table_walk<K, true, kStats>(p, u0.table_off + col, n_m, groups, m, W, map, s_rec + tid, act,
                                  counts, nrec, st_entries);
    else
      table_walk<K, false, kStats>(p, u0.table_off + col, n_m, groups, m, W, map, s_rec + tid, act,
                                   counts, nrec, st_entries);
    if (kStats) {
      const uint32_t ent = __reduce_add_sync(kFull, st_entries);
      const unsigned vq = __popc(__ballot_sync(kFull, valid));
      if ((tid & 31) == 0) {
        atomicAdd(&p.stats[kStatTableEntries], (unsigned long long)ent);
        atomicAdd(&p.stats[kStatTableQueries], (unsigned long long)vq * count);
      }
    }
    for (int b = 0; b < count; ++b) {
      const int unit = unit0 + b;
      const UnitDesc u = (b == 0) ? u0 : p.units[unit];
      const bool full = ((counts >> (8 * b)) & 0xffu) >= (uint32_t)K;
      if (kStats) {
        const unsigned fb = __popc(__ballot_sync(kFull, valid && !full));
        if ((tid & 31) == 0 && fb) atomicAdd(&p.stats[kStatTableFallbacks], (unsigned long long)fb);
      }
      int nb[E + 1];
      float dd[E + 1];
      // target values from the table (not when the neighbours are checked)
      bool tv = u.table_tv != 0 && p.table_pairs && p.dbg_nbr == nullptr;
      if (full || !valid) {
        // the first E+1 flagged ranks of the realization's records; their
        // indices and distances are read from the table (the stored distances
        // are the bits the epilogue would compute: the build used the same
        // rounding sequence and the same square root)
        const int nr = (int)((nrec >> (8 * b)) & 0xffu);
        const uint16_t* rec = s_rec + b * K * kThreads + tid;
        int ri = 0;
        uint32_t cur = valid ? rec[0] : 0u;
#pragma unroll
        for (int s2 = 0; s2 <= E; ++s2) {
          while ((cur & 0xffu) == 0u && ri + 1 < nr) cur = rec[(++ri) * kThreads];
          const uint32_t fl = cur & 0xffu;
          const int c = fl ? __ffs(fl) - 1 : 0;  // fl > 0 whenever the walk was full
          cur &= ~(1u << c);
          nb[s2] = 8 * (int)(cur >> 8) + c;  // the rank, for now
        }
        // the distances (not squared) and, when the table holds them, the
        // target's values at the neighbours (one 8-byte load each), else the
        // neighbours' indices (for the gather)
        auto at = [&](int rank) {
          return u0.table_off + (int64_t)(rank >> 2) * 4 * n_m + col + (rank & 3);
        };
        const float2* dv2 = reinterpret_cast<const float2*>(p.table_dist);
        if (tv) {
#pragma unroll
          for (int s2 = 0; s2 <= E; ++s2) {
            const float2 dv = valid ? __ldg(dv2 + at(nb[s2])) : make_float2(0.f, 0.f);
            dd[s2] = dv.x;
            nb[s2] = __float_as_int(dv.y);
          }
        } else {
#pragma unroll
          for (int s2 = 0; s2 <= E; ++s2) {
            const int64_t a2 = at(nb[s2]);
            dd[s2] = !valid ? 0.f : p.table_pairs ? __ldg(dv2 + a2).x : __ldg(p.table_dist + a2);
            nb[s2] = !valid ? 0
                            : (p.table_u16 ? (int)__ldg(static_cast<const uint16_t*>(p.table) + a2)
                                           : __ldg(static_cast<const int32_t*>(p.table) + a2));
          }
        }
      } else {
        // Rare: fewer than E+1 members among the R nearest points; scan the
        // library, keeping the E+1 smallest (distance, index) keys.
        const int32_t* lib = p.lib + u.lib_off;
        float q[E];
#pragma unroll
        for (int e = 0; e < E; ++e) q[e] = sj[m + off - e * tau];
        float kd[E + 1];
        int kl[E + 1];
#pragma unroll
        for (int s2 = 0; s2 <= E; ++s2) {
          kd[s2] = INFINITY;
          kl[s2] = INT_MAX;
        }
        for (int a = 0; a < L; ++a) {
          const int l = lib[a];
          if (abs(l - m) <= W) continue;
          const float d = d2_point<E>(sj, off, tau, q, l);
          if (key_less(d, l, kd[E], kl[E])) {
            int s2 = E;
            while (s2 > 0 && key_less(d, l, kd[s2 - 1], kl[s2 - 1])) {
              kd[s2] = kd[s2 - 1];
              kl[s2] = kl[s2 - 1];
              --s2;
            }
            kd[s2] = d;
            kl[s2] = l;
          }
        }
#pragma unroll
        for (int s2 = 0; s2 <= E; ++s2) {
          nb[s2] = min(max(kl[s2], 0), n_m - 1);  // in bounds however few points qualified
          dd[s2] = sqrt_hw(kd[s2]);
        }
        tv = false;  // gathered as for brute force
      }
      finish_tile<E, false, true>(p, u, unit, tile, m, valid, dd, nb, s_ring, meta, ring_n, nullptr,
                                  tv);
    }
  }
}

// kMinCtas CTAs per SM.  Four (64 registers a thread) for manifolds with a
// byte map: the walk waits on L2, and more resident warps hide more of it
// than the few spilled registers cost (the sweep's scan: 151 ms, 165 ms with
// three).  Three (80 registers) for longer manifolds (bitmap, one realization
// an item, tables beyond L2), which want the registers (the N = 10^5 series'
// scan: 110 ms, 120 ms with four).
template <int E, bool kStats, int kMinCtas>
__global__ void __launch_bounds__(kThreads, kMinCtas) knn_table_kernel(KnnParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ RingMeta s_meta[kRing];
  int ring_n = 0;  // staged prediction vectors (the same in every thread)
  for (int64_t round = 0;; ++round) {
    if (p.persistent) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(p.item_counter, 1u);
      __syncthreads();
    }
    const int it = p.persistent ? s_item : (round == 0 ? (int)blockIdx.x : INT_MAX);
    __syncthreads();
    if ((int64_t)it >= p.n_items) break;
    const WorkItem w = p.items[it];
    const UnitDesc u = p.units[w.unit];
    if (u.E != E || w.count < 1 || w.count > kTableGroup ||
        (w.count > 1 && u.n_m > kByteMapMax)) {
      if (threadIdx.x == 0) atomicOr(p.err, kErrBadUnit);
      continue;
    }
    process_table_item<E, kStats>(p, w.unit, w.count, w.tile, smem, s_meta, ring_n);
  }
  if (ring_n > 0) flush_ring(p, reinterpret_cast<const float*>(smem), s_meta, ring_n);
}

template <int E, bool kStats>
__global__ void __launch_bounds__(kThreads, 3) knn_fused_kernel(KnnParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ RingMeta s_meta[kRing];
  int ring_n = 0;  // staged prediction vectors (the same in every thread)
  for (int64_t round = 0;; ++round) {
    if (p.persistent) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(p.item_counter, 1u);
      __syncthreads();
    }
    const int it = p.persistent ? s_item : (round == 0 ? (int)blockIdx.x : INT_MAX);
    __syncthreads();
    if ((int64_t)it >= p.n_items) break;
    const WorkItem w = p.items[it];
    const UnitDesc u = p.units[w.unit];
    if (u.E != E) {
      if (threadIdx.x == 0) atomicOr(p.err, kErrBadUnit);
      continue;
    }
    if (p.variant[E] == 1)
      process_item<E, 1, kStats>(p, u, w.unit, w.tile, smem, s_meta, ring_n);
    else
      process_item<E, 0, kStats>(p, u, w.unit, w.tile, smem, s_meta, ring_n);
  }
  if (ring_n > 0)
    flush_ring(p, reinterpret_cast<const float*>(smem + kCoordBytes + kBufBytes), s_meta, ring_n);
}

}  // namespace

int knn_block_threads() { return kThreads; }

size_t knn_table_smem(int max_nm) {
  // every manifold of the launch fits: bytes up to kByteMapMax points, bits above
  const size_t bits = (size_t)((max_nm + 31) / 32) * 4;
  const size_t map = (max_nm <= kByteMapMax) ? (size_t)(max_nm + 3) / 4 * 4
                                             : (bits > (size_t)kByteMapMax ? bits : kByteMapMax);
  return (size_t)kRingBytes + (size_t)kRecBytes + map + 16;
}

#define CCM_FOR_E(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

cudaError_t knn_table_prepare() {
  // the largest bitmap any plan may need (manifolds up to kTableMaxNm points);
  // set once, so that plans of different sizes never lower it for each other
#define CCM_TPREP(EV)                                                             \
  for (const auto fn : {knn_table_kernel<EV, false, 4>, knn_table_kernel<EV, true, 4>,  \
                        knn_table_kernel<EV, false, 3>}) {                          \
    const cudaError_t e = cudaFuncSetAttribute(                                   \
        fn, cudaFuncAttributeMaxDynamicSharedMemorySize,                          \
        (int)knn_table_smem(kTableMaxNm));                                        \
    if (e != cudaSuccess) return e;                                               \
  }
  CCM_FOR_E(CCM_TPREP)
#undef CCM_TPREP
  return cudaSuccess;
}

// Launches whose manifolds exceed the byte map use the three-CTA kernels
// (the counting variant always the four-CTA ones).
cudaError_t knn_table_occupancy(int max_nm, int* ctas) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      ctas, max_nm > kByteMapMax ? knn_table_kernel<kMaxE, false, 3> : knn_table_kernel<kMaxE, false, 4>,
      kThreads, knn_table_smem(max_nm));
}

cudaError_t launch_knn_table(const KnnParams& p, int E, int max_nm, int grid, cudaStream_t s) {
#define CCM_TLAUNCH(EV)                                                           \
  if (E == EV) {                                                                  \
    if (p.stats)                                                                  \
      knn_table_kernel<EV, true, 4><<<grid, kThreads, knn_table_smem(max_nm), s>>>(p); \
    else if (max_nm > kByteMapMax)                                                \
      knn_table_kernel<EV, false, 3><<<grid, kThreads, knn_table_smem(max_nm), s>>>(p); \
    else                                                                          \
      knn_table_kernel<EV, false, 4><<<grid, kThreads, knn_table_smem(max_nm), s>>>(p); \
    return cudaGetLastError();                                                    \
  }
  CCM_FOR_E(CCM_TLAUNCH)
#undef CCM_TLAUNCH
  return cudaErrorInvalidValue;
}
int knn_queries_per_thread() { return 1; }

cudaError_t launch_obs(const float* series, const int32_t* order, const ObsJob* jobs,
                       int64_t n_jobs, int64_t n_tiles, double* obs, cudaStream_t s) {
  if (n_jobs <= 0 || n_tiles <= 0) return cudaSuccess;
  const int64_t want = (n_tiles + kThreads / 32 - 1) / (kThreads / 32);  // a warp per tile
  const int64_t blocks = want < 65536 ? want : 65536;
  obs_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(series, order, jobs, n_jobs, n_tiles, obs);
  return cudaGetLastError();
}

// One kernel per E (each keeps all its registers for that E's lists).

cudaError_t launch_knn(const KnnParams& p, int E, int grid, cudaStream_t s) {
#define CCM_LAUNCH(EV)                                                          \
  if (E == EV) {                                                                \
    if (p.stats)                                                                \
      knn_fused_kernel<EV, true><<<grid, kThreads, kSmemBytes, s>>>(p);         \
    else                                                                        \
      knn_fused_kernel<EV, false><<<grid, kThreads, kSmemBytes, s>>>(p);        \
    return cudaGetLastError();                                                  \
  }
  CCM_FOR_E(CCM_LAUNCH)
#undef CCM_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t knn_prepare() {
#define CCM_PREP(EV)                                                            \
  for (const auto fn : {knn_fused_kernel<EV, false>, knn_fused_kernel<EV, true>}) { \
    const cudaError_t e = cudaFuncSetAttribute(                                 \
        fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);           \
    if (e != cudaSuccess) return e;                                             \
  }
  CCM_FOR_E(CCM_PREP)
#undef CCM_PREP
  return cudaSuccess;
}

cudaError_t knn_occupancy(int E, int* ctas) {
#define CCM_OCC(EV)                                                             \
  if (E == EV)                                                                  \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, knn_fused_kernel<EV, false>,   \
                                                         kThreads, kSmemBytes);
  CCM_FOR_E(CCM_OCC)
#undef CCM_OCC
  return cudaErrorInvalidValue;
}

}  // namespace ccm
