// Distance indexing table (paper Sect. 3.2: a table of the sorted distances of
// every point, built once, from which the E+1 nearest neighbours of any
// subsample are read off instead of re-sorting all distances for every
// subsample; Sect. 3.2 and Fig. 2 describe it as a second pipeline that feeds
// the CCM transform).
//
// For one (library variable, E, tau) the table holds, for every query
// position pos of the query order, the R nearest manifold points of the query
// m = order[pos] over the WHOLE manifold, m itself left out (no neighbour
// list holds it), sorted by (FP32 squared distance, index), the same key the
// brute-force selection uses.  For a realization whose library is a subset of
// the manifold, the first E+1 table entries that are library members (outside
// the exclusion window) are exactly its E+1 nearest library neighbours:
// restricting a total order to a subset keeps its order.
//
// Layout: ranks in groups of four, table[table_off + (r/4) * 4*n_m + pos*4 +
// r%4], so that one 8-byte (16-bit entries) or 16-byte (32-bit) load gives a
// query four consecutive ranks and the 32 consecutive query positions of a
// warp read one group with one coalesced access; 16-bit entries when every
// manifold of the plan has fewer than 65536 points, else 32-bit.  A float
// array of the same layout holds each entry's distance (the square root the
// simplex weights take of the FP32 squared distance, computed the same way),
// so that the scan reads the E+1 distances it needs instead of recomputing
// them from E scattered coordinates each.
//
// Build: one warp per query position, one kernel per E (its registers follow
// that E).  A histogram of the top 11 bits of the
// FP32 bit patterns of all N_m squared distances finds the bin b1 holding rank
// R; a second pass collects every entry below b1 (all of them belong to the
// row) and the entries of b1; both are sorted by (bits, index) (bitonic sorts
// in shared memory), and the row is the entries below b1 followed by the
// first of b1.  When b1 holds more than kTableBoundary entries, two more radix
// passes (11, 10 bits) refine it to the exact R-th value T instead, a pass
// collects the entries below T and, in index order, the first ties, and one
// sort orders the R keys (bits << 32 | index).
#include <stdint.h>

#include <initializer_list>

#include "ccm_internal.h"

namespace ccm {
namespace {

constexpr int kTableWarps = 8;  // query positions per CTA
constexpr int kUnroll = 4;      // points per lane per distance-loop iteration
constexpr int kSampleMinNm = 32768;  // manifolds from this size build rows from a sample threshold
constexpr int kSampleStride = 8;     // the sample: every 8th manifold point
constexpr int kStageChunk = 2048;    // manifold points per staged series chunk
constexpr int kStageHalo = 1024;     // lag span (E-1)tau up to which the series is staged
constexpr int kTableBoundary = 512;  // boundary-bin entries sorted directly (else refined)

__host__ __device__ constexpr size_t table_warp_bytes(int rcap) {
  return (size_t)(rcap + kTableBoundary) * 8 > 2048 * 4 ? (size_t)(rcap + kTableBoundary) * 8
                                                        : (size_t)2048 * 4;
}
constexpr unsigned kFullMask = 0xffffffffu;

// FP32 squared distance from query coordinates q to manifold point x, in the
// fixed order (coordinate 0 a rounded product, then one fused multiply-add per
// coordinate): the same bits as the neighbour search computes.
template <int E>
__device__ __forceinline__ uint32_t d2_bits(const float* s, int off, int tau, const float (&q)[E],
                                            int x) {
  float diff = __fsub_rn(q[0], s[x + off]);
  float acc = __fmul_rn(diff, diff);
#pragma unroll
  for (int e = 1; e < E; ++e) {
    diff = __fsub_rn(q[e], s[x + off - e * tau]);
    acc = __fmaf_rn(diff, diff, acc);
  }
  return __float_as_uint(acc);  // d2 >= +0: unsigned order is numeric order
}

// Warp-wide scan of a histogram in shared memory: the bin holding the
// 1-based rank `rank`, and how many entries lie in the bins below it.
__device__ __forceinline__ void select_bin(const uint32_t* hist, int nbins, int rank, int* bin_out,
                                           uint32_t* before_out, uint32_t* count_out) {
  const int lane = threadIdx.x & 31;
  const int chunk = nbins / 32;  // each lane owns a contiguous chunk of bins
  uint32_t mine = 0u;
  for (int b = 0; b < chunk; ++b) mine += hist[lane * chunk + b];
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned hit = __ballot_sync(kFullMask, incl >= (uint32_t)rank);
  const int owner = __ffs(hit) - 1;  // exists: the histogram holds >= rank entries
  uint32_t before = incl - mine, count = 0u;
  int bin = 0;
  if (lane == owner) {
    for (int b = 0; b < chunk; ++b) {
      const uint32_t h = hist[lane * chunk + b];
      if (before + h >= (uint32_t)rank) {
        bin = lane * chunk + b;
        count = h;
        break;
      }
      before += h;
    }
  }
  *bin_out = __shfl_sync(kFullMask, bin, owner);
  *before_out = __shfl_sync(kFullMask, before, owner);
  *count_out = __shfl_sync(kFullMask, count, owner);
}

// Ascending bitonic sort of n (a power of two, >= 32) keys by one warp.  Each
// stage has n/2 compare-exchange pairs (i, i + jj), i the t-th index with bit
// jj clear: every lane takes whole pairs.
__device__ __forceinline__ void warp_bitonic(unsigned long long* keys, int n) {
  const int lane = threadIdx.x & 31;
  const int half = n >> 1;
  for (int k = 2; k <= n; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int t = lane; t < half; t += 32) {
        const int i = 2 * t - (t & (jj - 1));
        const unsigned long long a = keys[i], b = keys[i + jj];
        if ((a > b) == ((i & k) == 0)) {
          keys[i] = b;
          keys[i + jj] = a;
        }
      }
      __syncwarp();
    }
  }
}

// The same distance with the coordinates read from a staged chunk of the
// series: stage[j] = s[base + j], xl = x - base.
template <int E>
__device__ __forceinline__ uint32_t d2_bits_staged(const float* stage, int off, int tau,
                                                   const float (&q)[E], int xl) {
  float diff = __fsub_rn(q[0], stage[xl + off]);
  float acc = __fmul_rn(diff, diff);
#pragma unroll
  for (int e = 1; e < E; ++e) {
    diff = __fsub_rn(q[e], stage[xl + off - e * tau]);
    acc = __fmaf_rn(diff, diff, acc);
  }
  return __float_as_uint(acc);
}

// One row (query position pos) of a table, by one warp.  `row`: pos is a
// query of the job (a warp without one takes part in the block-wide staging
// of the sampled path only); `stage`: shared memory for kStageChunk + kStageHalo
// series values, or null.
template <int E>
__device__ void build_row(const float* s, const TableJob& jb, int pos, bool row,
                          const int32_t* order, void* table, float* table_dist, int pairs,
                          const float* tv_series, int u16,
                          uint32_t* hist, unsigned long long* keys, unsigned long long* bnd,
                          uint32_t* cnt, int region_keys, float* stage) {
  const int lane = threadIdx.x & 31;
  const unsigned below_lane = (1u << lane) - 1u;
  const int n_m = jb.n_m, tau = jb.tau, off = (E - 1) * tau, R = jb.R;
  const int m = order[jb.order_off + (row ? pos : 0)];
  float q[E];
#pragma unroll
  for (int e = 0; e < E; ++e) q[e] = s[m + off - e * tau];
  auto key_of = [](uint32_t bits, int x) { return ((unsigned long long)bits << 32) | (unsigned)x; };

  // Long manifolds: one collecting pass below a threshold estimated from a
  // sample of one point in kSampleStride, taken as runs of 32 consecutive
  // points spread over the manifold (coalesced loads; two histogram levels give
  // the sample's k-th smallest distance to 21 bits; k is chosen so that about
  // (R + C)/2 of all points fall below it, C the largest power of two the
  // warp's key region holds), then one sort of the collected keys.  If the
  // count misses [R, C] the exact passes below run instead.  The collecting
  // pass reads the series through shared memory, chunk by chunk, staged once
  // for the CTA's eight rows (the decision is the same for the whole CTA).
  bool sampled = false;
  int C = 1;
  while (2 * C <= region_keys) C <<= 1;
  if (n_m >= kSampleMinNm && R < C) {
   uint32_t T = 0u;
   if (row) {
    const int runs = n_m / (32 * kSampleStride);           // whole runs inside the manifold
    const int S = runs * 32;
    const int k = (int)(((int64_t)(R + C) / 2 * S + n_m - 1) / n_m);  // >= 1, < S
    for (int b = lane; b < 2048; b += 32) hist[b] = 0u;
    __syncwarp();
    // sample point i: run i/32 (runs kSampleStride*32 points apart), offset i%32
    auto sample_x = [](int i) { return (i >> 5) * (32 * kSampleStride) + (i & 31); };
    // runs are far apart (L2 latency): four runs' loads in flight per lane
    for (int i0 = 0; i0 < S; i0 += 32 * kUnroll) {  // S is a multiple of 32: whole warps
      uint32_t b[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + 32 * u + lane;
        b[u] = (i < S) ? d2_bits<E>(s, off, tau, q, sample_x(i)) >> 21 : 0xffffffffu;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        // lanes that share a bin add once (the coarse bins are crowded)
        const unsigned same = __match_any_sync(kFullMask, b[u]);
        if (b[u] != 0xffffffffu && lane == __ffs(same) - 1)
          atomicAdd(&hist[b[u]], (uint32_t)__popc(same));
      }
    }
    __syncwarp();
    int bs1, bs2;
    uint32_t bef1, c1, bef2, c2;
    select_bin(hist, 2048, k, &bs1, &bef1, &c1);
    __syncwarp();
    for (int b = lane; b < 1024; b += 32) hist[b] = 0u;
    __syncwarp();
    for (int i0 = lane; i0 < S; i0 += 32 * kUnroll) {
      uint32_t bits[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + 32 * u;
        bits[u] = (i < S) ? d2_bits<E>(s, off, tau, q, sample_x(i)) : 0xffffffffu;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if ((bits[u] >> 21) == (uint32_t)bs1) atomicAdd(&hist[(bits[u] >> 11) & 1023u], 1u);
    }
    __syncwarp();
    select_bin(hist, 1024, k - (int)bef1, &bs2, &bef2, &c2);
    T = ((uint32_t)bs1 << 21) | ((uint32_t)bs2 << 11) | 0x7ffu;
   }
    if (lane == 0) cnt[0] = 0u;
    __syncwarp();
    if (stage) {
      for (int base = 0; base < n_m; base += kStageChunk) {
        const int len = min(kStageChunk, n_m - base);
        __syncthreads();  // the previous chunk has been read
        for (int i = threadIdx.x; i < len + off; i += blockDim.x) stage[i] = s[base + i];
        __syncthreads();
        if (row) {
          for (int x0 = lane; x0 < len; x0 += 32 * kUnroll) {
            uint32_t bits[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
              const int xl = x0 + 32 * u;
              bits[u] = (xl < len) ? d2_bits_staged<E>(stage, off, tau, q, xl) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
              if (bits[u] <= T && x0 + 32 * u < len && base + x0 + 32 * u != m) {
                const uint32_t at = atomicAdd(&cnt[0], 1u);
                if (at < (uint32_t)C) keys[at] = key_of(bits[u], base + x0 + 32 * u);
              }
            }
          }
        }
      }
    } else if (row) {
    for (int x0 = lane; x0 < n_m; x0 += 32 * kUnroll) {
      uint32_t bits[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int x = x0 + 32 * u;
        bits[u] = (x < n_m) ? d2_bits<E>(s, off, tau, q, x) : 0xffffffffu;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (bits[u] <= T && x0 + 32 * u < n_m && x0 + 32 * u != m) {
          const uint32_t at = atomicAdd(&cnt[0], 1u);
          if (at < (uint32_t)C) keys[at] = key_of(bits[u], x0 + 32 * u);
        }
      }
    }
    }
    __syncwarp();
    const int c = (int)cnt[0];
    if (row && c >= R && c <= C) {
      int p2 = 32;
      while (p2 < c) p2 <<= 1;
      for (int i = c + lane; i < p2; i += 32) keys[i] = ~0ull;
      __syncwarp();
      warp_bitonic(keys, p2);
      sampled = true;
    }
    __syncwarp();
  }
  if (!row) return;
  if (!sampled) {
  // Pass 1: histogram of the top 11 bits (non-negative floats order like
  // their bit patterns); the bin b1 holding rank R.
  for (int b = lane; b < 2048; b += 32) hist[b] = 0u;
  __syncwarp();
  for (int x = lane; x < n_m; x += 32) atomicAdd(&hist[d2_bits<E>(s, off, tau, q, x) >> 21], 1u);
  __syncwarp();
  // m itself was counted: its squared distance is exactly 0 (bin 0)
  if (lane == 0) hist[0] -= 1u;
  __syncwarp();
  int b1;
  uint32_t below1, in_b1;
  select_bin(hist, 2048, R, &b1, &below1, &in_b1);
  __syncwarp();

  if (in_b1 <= (uint32_t)kTableBoundary) {
    // Pass 2: every entry below b1 is a row entry; the entries of b1 are
    // sorted and the first R - below1 of them complete the row.
    // positions by shared-memory atomics (the entries are rare): no warp vote
    // in the loop, so consecutive iterations' loads overlap; both lists are
    // sorted by their full keys below, so the arrival order does not matter
    if (lane == 0) cnt[0] = cnt[1] = 0u;
    __syncwarp();
    for (int x = lane; x < n_m; x += 32) {
      const uint32_t bits = d2_bits<E>(s, off, tau, q, x);
      const uint32_t bin = (x != m) ? bits >> 21 : 0xffffffffu;
      if (bin < (uint32_t)b1) keys[atomicAdd(&cnt[0], 1u)] = key_of(bits, x);
      else if (bin == (uint32_t)b1) bnd[atomicAdd(&cnt[1], 1u)] = key_of(bits, x);
    }
    __syncwarp();
    const uint32_t nb = cnt[1];
    int p2 = 32;
    while (p2 < (int)nb) p2 <<= 1;
    for (int i = (int)nb + lane; i < p2; i += 32) bnd[i] = ~0ull;
    __syncwarp();
    warp_bitonic(bnd, p2);
    // every entry below b1 precedes every entry of b1: sort only those below
    // (padded to a power of two), then append the boundary bin's first ones
    int pl = 32;
    while (pl < (int)below1) pl <<= 1;
    for (int i = (int)below1 + lane; i < pl; i += 32) keys[i] = ~0ull;
    __syncwarp();
    warp_bitonic(keys, pl);
    for (int i = lane; i < R - (int)below1; i += 32) keys[below1 + i] = bnd[i];
  } else {
    // A crowded boundary bin: refine it with two more radix passes (11 and 10
    // bits) to the exact R-th bit pattern T and how many entries equal to T
    // are taken, then collect in index order.
    uint32_t prefix = (uint32_t)b1 << 21, mask = 0x7ffu << 21;
    int rank = R - (int)below1;
    for (int pass = 1; pass < 3; ++pass) {
      const int sh = (pass == 1) ? 10 : 0;
      const int nbins = (pass == 2) ? 1024 : 2048;
      const uint32_t dm = (uint32_t)nbins - 1u;
      for (int b = lane; b < nbins; b += 32) hist[b] = 0u;
      __syncwarp();
      for (int x = lane; x < n_m; x += 32) {
        const uint32_t bits = d2_bits<E>(s, off, tau, q, x);
        if ((bits & mask) == prefix) atomicAdd(&hist[(bits >> sh) & dm], 1u);
      }
      __syncwarp();
      if (lane == 0 && prefix == 0u) hist[0] -= 1u;  // m itself (bits 0) was counted
      __syncwarp();
      int bin;
      uint32_t before, cnt;
      select_bin(hist, nbins, rank, &bin, &before, &cnt);
      prefix |= (uint32_t)bin << sh;
      mask |= dm << sh;
      rank -= (int)before;
      __syncwarp();
    }
    const uint32_t T = prefix;   // bit pattern of the R-th smallest squared distance
    const int take_ties = rank;  // entries equal to T to take, lowest index first
    const int n_less = R - take_ties;
    int less_seen = 0, ties_seen = 0;
    for (int base = 0; base < n_m; base += 32) {
      const int x = base + lane;
      const uint32_t bits = (x < n_m) ? d2_bits<E>(s, off, tau, q, x) : 0xffffffffu;
      const bool less = (x < n_m) && x != m && bits < T;
      const bool tie = (x < n_m) && x != m && bits == T;
      const unsigned lm = __ballot_sync(kFullMask, less);
      const unsigned tm = __ballot_sync(kFullMask, tie);
      if (less) keys[less_seen + __popc(lm & below_lane)] = key_of(bits, x);
      const int tr = ties_seen + __popc(tm & below_lane);
      if (tie && tr < take_ties) keys[n_less + tr] = key_of(bits, x);
      less_seen += __popc(lm);
      ties_seen += __popc(tm);
    }
    int rcap = 32;  // this row's sort size: the power of two at or above R
    while (rcap < R) rcap <<= 1;
    for (int i = R + lane; i < rcap; i += 32) keys[i] = ~0ull;
    __syncwarp();
    warp_bitonic(keys, rcap);
  }
  }
  __syncwarp();
  const int64_t base = jb.table_off + (int64_t)pos * 4;
  // each entry's distance (the epilogue's square root), beside it; with pairs,
  // together with the target's value at the entry's point (what the
  // prediction weighs; 0 in a table without a target)
  for (int r = lane; r < R; r += 32) {
    const int64_t at = base + (int64_t)(r >> 2) * 4 * n_m + (r & 3);
    const float d = sqrt_hw(__uint_as_float((uint32_t)(keys[r] >> 32)));
    if (pairs)
      reinterpret_cast<float2*>(table_dist)[at] =
          make_float2(d, jb.tv_i >= 0 ? tv_series[(int)(keys[r] & 0xffffffffu) + off] : 0.f);
    else
      table_dist[at] = d;
  }
  if (u16) {
    uint16_t* out = static_cast<uint16_t*>(table) + base;
    for (int r = lane; r < R; r += 32)
      out[(int64_t)(r >> 2) * 4 * n_m + (r & 3)] = (uint16_t)(keys[r] & 0xffffu);
  } else {
    int32_t* out = static_cast<int32_t*>(table) + base;
    for (int r = lane; r < R; r += 32)
      out[(int64_t)(r >> 2) * 4 * n_m + (r & 3)] = (int32_t)(keys[r] & 0xffffffffu);
  }
  __syncwarp();
}

// kMinCtas CTAs per SM: 2 (128 registers) for the exact two-pass build of
// short manifolds, 3 for the sampled single pass of long ones, whose loads
// want more warps in flight (measured: the sweep's tables 63 vs 68 ms with 3,
// the N = 10^5 series' 203 vs 185 ms).
template <int E, int kMinCtas>
__global__ void __launch_bounds__(kTableWarps * 32, kMinCtas)
table_build_kernel(const float* series, const TableJob* jobs, const int32_t* order, void* table,
                   float* table_dist, int pairs, int u16, int rcap, int staged) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_cnt[kTableWarps][2];  // per warp: entries below b1, entries of b1
  const TableJob jb = jobs[blockIdx.y];
  if (jb.E != E) return;  // the same job for the whole CTA
  const int warp = threadIdx.x >> 5;
  const int pos = blockIdx.x * kTableWarps + warp;
  if (blockIdx.x * kTableWarps >= jb.n_m) return;  // the whole CTA past this job's rows
  // per warp: the 2048 histogram bins, overlapping the rcap row keys and the
  // kTableBoundary keys of the boundary bin
  unsigned char* mine = smem + warp * table_warp_bytes(rcap);
  uint32_t* hist = reinterpret_cast<uint32_t*>(mine);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(mine);
  unsigned long long* bnd = keys + rcap;
  const float* s = series + jb.series_off + (int64_t)jb.j * jb.n;
  // staged collecting pass from E = 5 (below that the chunk barriers cost
  // more than the loads they save); the launch reserved the space
  float* stage = (staged && (E - 1) * jb.tau <= kStageHalo)
                     ? reinterpret_cast<float*>(smem + kTableWarps * table_warp_bytes(rcap))
                     : nullptr;
  const float* tv_series = series + jb.series_off + (int64_t)(jb.tv_i >= 0 ? jb.tv_i : 0) * jb.n;
  build_row<E>(s, jb, pos, pos < jb.n_m, order, table, table_dist, pairs, tv_series, u16, hist,
               keys, bnd,
               s_cnt[warp], (int)(table_warp_bytes(rcap) / 8), stage);
}

size_t table_smem(int rcap, bool staged) {
  return (size_t)kTableWarps * table_warp_bytes(rcap) +
         (staged ? (kStageChunk + kStageHalo) * sizeof(float) : 0);
}

}  // namespace

#define CCM_FOR_E(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

cudaError_t table_prepare() {
#define CCM_TBPREP(EV)                                                                   \
  for (const auto fn : {table_build_kernel<EV, 2>, table_build_kernel<EV, 3>}) {         \
    const cudaError_t e = cudaFuncSetAttribute(                                          \
        fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)table_smem(kTableMaxR, true)); \
    if (e != cudaSuccess) return e;                                                      \
  }
  CCM_FOR_E(CCM_TBPREP)
#undef CCM_TBPREP
  return cudaSuccess;
}

cudaError_t launch_table_build(const float* series, const TableJob* jobs, int64_t n_jobs, int E,
                               int max_nm, int max_R, const int32_t* order, void* table,
                               float* table_dist, int table_pairs, int table_u16, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  int rcap = 32;
  while (rcap < max_R) rcap <<= 1;
  if (rcap > kTableMaxR) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((max_nm + kTableWarps - 1) / kTableWarps), (unsigned)n_jobs);
  const int staged = (E >= 5 && max_nm >= kSampleMinNm) ? 1 : 0;
#define CCM_TBLAUNCH(EV)                                                                 \
  if (E == EV) {                                                                         \
    if (max_nm >= kSampleMinNm)                                                          \
      table_build_kernel<EV, 3><<<grid, kTableWarps * 32, table_smem(rcap, staged), s>>>( \
          series, jobs, order, table, table_dist, table_pairs, table_u16, rcap, staged);   \
    else                                                                                 \
      table_build_kernel<EV, 2><<<grid, kTableWarps * 32, table_smem(rcap, staged), s>>>( \
          series, jobs, order, table, table_dist, table_pairs, table_u16, rcap, staged);   \
    return cudaGetLastError();                                                           \
  }
  CCM_FOR_E(CCM_TBLAUNCH)
#undef CCM_TBLAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace ccm
