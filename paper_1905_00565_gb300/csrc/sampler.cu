// Library sampler: r random libraries of L manifold points, drawn without
// replacement (paper Sect. 1: r random subsamples of size L; Sect. 3.1: the
// pipeline input is a set of subsamples per (tau, E, L)).
//
// Random-key selection: manifold point m of unit (j, E, tau, L, k) gets the
// 64-bit key (hi32(w0) << 32) | m, where w0 is word 0 of Philox4x64-10 at
// counter (m, k, L, (j<<16)|(E<<8)|tau) under key (seed, 0).  The library is
// the L points with the smallest keys, written in ascending m.  Keys are
// distinct, so the selection is a pure function of the counter.
//
// One CTA per unit.  The high halves h(m) are computed once into shared memory
// (or recomputed per pass when N_m is too large), an 8-bit radix select over
// four passes finds the L-th smallest key (h*, and how many of the h == h*
// points, smallest m first, are taken).  An in-order block compaction over m
// finds the largest tie taken (and writes the checking copy, ascending m); a
// second one over the unit's query order writes the library in query order,
// the order the neighbour search visits it in (spatially coherent runs).
#include "ccm_internal.h"

namespace ccm {
namespace {

// Philox4x64-10 (Salmon et al., SC'11): ten rounds, two 64x64->128 products per
// round, round keys bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint64_t philox_word0(uint64_t c0, uint64_t c1, uint64_t c2,
                                                 uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return c0;
}

__device__ __forceinline__ uint32_t key_hi(const UnitDesc& u, int m) {
  const uint64_t c3 = ((uint64_t)u.j << 16) | ((uint64_t)u.E << 8) | (uint64_t)u.tau;
  return (uint32_t)(philox_word0((uint64_t)m, (uint64_t)u.k, (uint64_t)u.L, c3, u.seed, 0) >> 32);
}

// Exclusive block scan of one uint32 per thread; returns the block total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* excl, uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = (lane < nwarps) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nwarps) warp_tot[lane] = t;  // inclusive prefix of warp totals
  }
  __syncthreads();
  const uint32_t before = (warp > 0) ? warp_tot[warp - 1] : 0u;
  *excl = before + x - v;
  const uint32_t total = warp_tot[nwarps - 1];
  __syncthreads();
  return total;
}

template <bool kInSmem>
__global__ void __launch_bounds__(kSamplerThreads)
sampler_kernel(SamplerParams p, int64_t first_unit) {
  extern __shared__ uint32_t s_keys[];
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_prefix, s_rank;
  __shared__ int s_mtie;

  const int64_t uidx = first_unit + blockIdx.x;
  const UnitDesc u = p.units[uidx];
  const int n_m = u.n_m, L = u.L;
  if (L < 1 || L > n_m) {
    if (threadIdx.x == 0) atomicOr(p.err, kErrSampler);
    return;
  }
  if (kInSmem) {
    for (int m = threadIdx.x; m < n_m; m += blockDim.x) s_keys[m] = key_hi(u, m);
  }
  if (threadIdx.x == 0) {
    s_prefix = 0u;
    s_rank = (uint32_t)L;  // 1-based rank still to find within the current prefix
    s_mtie = -1;
  }
  uint32_t mask = 0u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) s_hist[b] = 0u;
    __syncthreads();
    const uint32_t prefix = s_prefix;
    for (int m = threadIdx.x; m < n_m; m += blockDim.x) {
      const uint32_t h = kInSmem ? s_keys[m] : key_hi(u, m);
      if ((h & mask) == prefix) atomicAdd(&s_hist[(h >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t rank = s_rank, cum = 0u;
      int b = 0;
      for (; b < 256; ++b) {
        if (cum + s_hist[b] >= rank) break;
        cum += s_hist[b];
      }
      s_prefix = prefix | ((uint32_t)b << shift);
      s_rank = rank - cum;
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  const uint32_t hstar = s_prefix;   // high half of the L-th smallest key
  const uint32_t take_ties = s_rank; // points with h == h* to take, smallest m first

  // In-order compaction over contiguous chunks of m.
  const int chunk = (n_m + blockDim.x - 1) / blockDim.x;
  const int m0 = min(n_m, (int)threadIdx.x * chunk), m1 = min(n_m, m0 + chunk);
  uint32_t n_less = 0u, n_tie = 0u;
  for (int m = m0; m < m1; ++m) {
    const uint32_t h = kInSmem ? s_keys[m] : key_hi(u, m);
    n_less += (h < hstar);
    n_tie += (h == hstar);
  }
  uint32_t tie_before;
  block_exclusive_scan(n_tie, &tie_before, s_warp);
  const uint32_t ties_here =
      (tie_before >= take_ties) ? 0u : min(n_tie, take_ties - tie_before);
  uint32_t out_before;
  const uint32_t total = block_exclusive_scan(n_less + ties_here, &out_before, s_warp);
  if (total != (uint32_t)L) {
    if (threadIdx.x == 0) atomicOr(p.err, kErrSampler);
    return;
  }
  uint32_t w = out_before, tie_seen = tie_before;
  for (int m = m0; m < m1; ++m) {
    const uint32_t h = kInSmem ? s_keys[m] : key_hi(u, m);
    bool take = h < hstar;
    if (h == hstar) {
      take = tie_seen < take_ties;
      if (take && tie_seen + 1 == take_ties) s_mtie = m;  // the last tie taken
      ++tie_seen;
    }
    if (take) {
      if (p.dbg_lib)  // checking copy, once per target of this library
        for (int t = 0; t < u.n_targets; ++t)
          p.dbg_lib[p.targets[u.tgt_off + t].lib_dbg_off + w] = m;
      ++w;
    }
  }
  __syncthreads();
  const int mtie = s_mtie;  // members: h < h*, or h == h* and m <= mtie

  // The library in query order: compaction over contiguous chunks of positions.
  const int32_t* ord = p.order + u.order_off;
  uint32_t n_mem = 0u;
  for (int q = m0; q < m1; ++q) {
    const int m = ord[q];
    const uint32_t h = kInSmem ? s_keys[m] : key_hi(u, m);
    n_mem += (h < hstar || (h == hstar && m <= mtie));
  }
  uint32_t pos_before;
  const uint32_t total2 = block_exclusive_scan(n_mem, &pos_before, s_warp);
  if (total2 != (uint32_t)L) {
    if (threadIdx.x == 0) atomicOr(p.err, kErrSampler);
    return;
  }
  int32_t* out = p.lib + u.lib_off;
  w = pos_before;
  for (int q = m0; q < m1; ++q) {
    const int m = ord[q];
    const uint32_t h = kInSmem ? s_keys[m] : key_hi(u, m);
    if (h < hstar || (h == hstar && m <= mtie)) out[w++] = m;
  }
}

}  // namespace

cudaError_t sampler_prepare() {
  return cudaFuncSetAttribute(sampler_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kSamplerSmemKeys * sizeof(uint32_t)));
}

cudaError_t launch_sampler(const SamplerParams& p, int64_t first_unit, int64_t count, int max_nm,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (max_nm <= kSamplerSmemKeys) {
    const size_t smem = (size_t)max_nm * sizeof(uint32_t);
    for (int64_t off = 0; off < count; off += 0x7fffffff) {
      const unsigned grid = (unsigned)((count - off) < 0x7fffffff ? (count - off) : 0x7fffffff);
      sampler_kernel<true><<<grid, kSamplerThreads, smem, s>>>(p, first_unit + off);
    }
  } else {
    for (int64_t off = 0; off < count; off += 0x7fffffff) {
      const unsigned grid = (unsigned)((count - off) < 0x7fffffff ? (count - off) : 0x7fffffff);
      sampler_kernel<false><<<grid, kSamplerThreads, 0, s>>>(p, first_unit + off);
    }
  }
  return cudaGetLastError();
}

}  // namespace ccm
