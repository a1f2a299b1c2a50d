// Library sampler: r random libraries of L manifold points, drawn without
// replacement (paper Sect. 1: r random subsamples of size L; Sect. 3.1: the
// pipeline input is a set of subsamples per (tau, E, L)).
//
// Random-key selection: manifold point m of unit (j, E, tau, L, k) gets the
// 64-bit key (v << 32) | m, where v is 32-bit half number m mod 8 of the
// Philox4x64-10 block at counter (floor(m/8), k, L, (j<<16)|(E<<8)|tau) under
// key (seed, 0), the halves numbered hi(w0), lo(w0), hi(w1), ..., lo(w3): one
// block gives the keys of eight consecutive points.  The library is the L
// points with the smallest keys, written in ascending m.  Keys are distinct,
// so the selection is a pure function of the counter.
//
// One CTA per unit.  The high halves h(m) are computed once into shared memory
// (or recomputed per pass when N_m is too large), an 8-bit radix select over
// four passes (bins scanned by one warp) finds the L-th smallest key (h*, and
// how many of the h == h* points, smallest m first, are taken; when some ties
// are left out, one warp finds the last tie taken).  A warp-by-warp stable
// compaction over the unit's query order writes the library in query order,
// the order the neighbour search visits it in (spatially coherent runs); the
// checking copy is compacted in ascending m.
#include "ccm_internal.h"

namespace ccm {
namespace {

// Philox4x64-10 (Salmon et al., SC'11): ten rounds, two 64x64->128 products per
// round, round keys bumped by the Weyl constants between rounds.  Writes the
// four output words.
__device__ __forceinline__ void philox_block(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                             uint64_t k0, uint64_t k1, uint64_t (&w)[4]) {
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
  w[0] = c0;
  w[1] = c1;
  w[2] = c2;
  w[3] = c3;
}

// The Philox block holding the keys of points 8b .. 8b+7.
__device__ __forceinline__ void key_block(const UnitDesc& u, int b, uint64_t (&w)[4]) {
  const uint64_t c3 = ((uint64_t)u.j << 16) | ((uint64_t)u.E << 8) | (uint64_t)u.tau;
  philox_block((uint64_t)b, (uint64_t)u.k, (uint64_t)u.L, c3, u.seed, 0, w);
}

// 32-bit half number i (0..7) of a block: hi(w0), lo(w0), hi(w1), ..., lo(w3).
__device__ __forceinline__ uint32_t block_half(const uint64_t (&w)[4], int i) {
  const int q = i >> 1;
  const uint64_t x = (q == 0) ? w[0] : (q == 1) ? w[1] : (q == 2) ? w[2] : w[3];
  return (i & 1) ? (uint32_t)x : (uint32_t)(x >> 32);
}

// The high half of point m's key (one block per call).
__device__ __forceinline__ uint32_t key_hi(const UnitDesc& u, int m) {
  uint64_t w[4];
  key_block(u, m >> 3, w);
  return block_half(w, m & 7);
}

// Stable compaction of the members among positions [0, n) by the whole block,
// warp by warp: warp w walks its contiguous segment 32 positions at a time
// (coalesced reads), counts members with a ballot, and after a block scan of
// the warp counts writes them in position order.  item(q) gives the manifold
// point at position q; is_member(m) decides membership.  `out` has room for
// `expect` entries: when the members number anything else (a sampler fault)
// nothing is compacted and out[0..expect) is filled with point 0 instead, so
// that later kernels reading the library stay in bounds.
template <typename Item, typename Member>
__device__ uint32_t block_compact(int n, Item item, Member is_member, int32_t* out,
                                  uint32_t expect, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int seg = ((n + nwarps - 1) / nwarps + 31) / 32 * 32;
  const int q0 = min(n, warp * seg), q1 = min(n, q0 + seg);
  uint32_t count = 0u;
  for (int q = q0 + lane; q - lane < q1; q += 32) {
    const bool mem = q < q1 && is_member(item(q));
    count += __popc(__ballot_sync(0xffffffffu, mem));
  }
  if (lane == 0) s_warp[warp] = count;
  __syncthreads();
  uint32_t base = 0u, total = 0u;
  for (int w = 0; w < nwarps; ++w) {
    base += (w < warp) ? s_warp[w] : 0u;
    total += s_warp[w];
  }
  __syncthreads();
  if (total != expect) {
    for (uint32_t q = threadIdx.x; q < expect; q += blockDim.x) out[q] = 0;
    return total;
  }
  for (int q = q0 + lane; q - lane < q1; q += 32) {
    const int m = q < q1 ? item(q) : 0;
    const bool mem = q < q1 && is_member(m);
    const unsigned bal = __ballot_sync(0xffffffffu, mem);
    if (mem) out[base + __popc(bal & ((1u << lane) - 1u))] = m;
    base += __popc(bal);
  }
  return total;
}

template <bool kInSmem>
__global__ void __launch_bounds__(kSamplerThreads)
sampler_kernel(SamplerParams p, int64_t first_unit) {
  extern __shared__ __align__(16) uint32_t s_keys[];
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_prefix, s_rank, s_neq;
  __shared__ int s_mtie;

  const int64_t uidx = first_unit + blockIdx.x;
  const UnitDesc u = p.units[uidx];
  const int n_m = u.n_m, L = u.L;
  const int lane = threadIdx.x & 31;
  if (L < 1 || L > n_m) {
    if (threadIdx.x == 0) atomicOr(p.err, kErrSampler);
    return;
  }
  const int n_blocks = (n_m + 7) >> 3;
  if (kInSmem) {  // the key array is padded to whole blocks of eight
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) {
      uint64_t w[4];
      key_block(u, b, w);
      uint4* dst = reinterpret_cast<uint4*>(s_keys + 8 * b);
      dst[0] = make_uint4(block_half(w, 0), block_half(w, 1), block_half(w, 2), block_half(w, 3));
      dst[1] = make_uint4(block_half(w, 4), block_half(w, 5), block_half(w, 6), block_half(w, 7));
    }
  }
  if (threadIdx.x == 0) {
    s_prefix = 0u;
    s_rank = (uint32_t)L;  // 1-based rank still to find within the current prefix
  }
  uint32_t mask = 0u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) s_hist[b] = 0u;
    __syncthreads();
    const uint32_t prefix = s_prefix;
    if (kInSmem) {
      for (int m = threadIdx.x; m < n_m; m += blockDim.x) {
        const uint32_t h = s_keys[m];
        if ((h & mask) == prefix) atomicAdd(&s_hist[(h >> shift) & 255u], 1u);
      }
    } else {  // recomputed, a block of eight keys per call
      for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) {
        uint64_t w[4];
        key_block(u, b, w);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t h = block_half(w, i);
          if (8 * b + i < n_m && (h & mask) == prefix) atomicAdd(&s_hist[(h >> shift) & 255u], 1u);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // the bin holding rank s_rank: lane l sums bins 8l..8l+7, then a warp scan
      const uint32_t rank = s_rank;
      uint32_t mine = 0u;
#pragma unroll
      for (int b = 0; b < 8; ++b) mine += s_hist[lane * 8 + b];
      uint32_t incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, incl >= rank);
      const int owner = __ffs(hit) - 1;  // exists: the histogram holds >= rank keys
      if (lane == owner) {
        uint32_t cum = incl - mine;
        int b = lane * 8;
        for (; b < lane * 8 + 7; ++b) {
          if (cum + s_hist[b] >= rank) break;
          cum += s_hist[b];
        }
        s_prefix = prefix | ((uint32_t)b << shift);
        s_rank = rank - cum;
        s_neq = s_hist[b];  // after the last pass: the keys equal to h*
      }
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  const uint32_t hstar = s_prefix;   // high half of the L-th smallest key
  const uint32_t take_ties = s_rank; // points with h == h* to take, smallest m first

  // Members: h < h*, or h == h* and m <= mtie (the last tie taken).  Almost
  // always every tie is taken; otherwise warp 0 finds the take_ties-th tie.
  if (threadIdx.x < 32) {
    int mtie = 0x7fffffff;
    if (take_ties < s_neq) {
      uint32_t seen = 0u;
      mtie = -1;
      for (int m0 = 0; m0 < n_m && mtie < 0; m0 += 32) {
        const int m = m0 + lane;
        const bool tie = m < n_m && (kInSmem ? s_keys[m] : key_hi(u, m)) == hstar;
        const unsigned bal = __ballot_sync(0xffffffffu, tie);
        if (seen + __popc(bal) >= take_ties) {
          unsigned b = bal;
          for (uint32_t k = seen + 1; k < take_ties; ++k) b &= b - 1u;  // drop earlier ties
          mtie = m0 + __ffs(b) - 1;
        }
        seen += __popc(bal);
      }
    }
    if (lane == 0) s_mtie = mtie;
  }
  __syncthreads();
  const int mtie = s_mtie;
  auto is_member = [&](int m) {
    const uint32_t h = kInSmem ? s_keys[m] : key_hi(u, m);
    return h < hstar || (h == hstar && m <= mtie);
  };
  // The library in query order (the order the neighbour search visits it in).
  const int32_t* ord = p.order + u.order_off;
  const uint32_t total = block_compact(n_m, [&](int q) { return ord[q]; }, is_member,
                                       p.lib + u.lib_off, (uint32_t)L, s_warp);
  if (total != (uint32_t)L) {  // not a permutation, or a lost tie: report, never guess
    if (threadIdx.x == 0) atomicOr(p.err, kErrSampler);
    return;
  }
  if (p.dbg_lib) {  // checking copy in ascending m, once per target of this library
    for (int t = 0; t < u.n_targets; ++t) {
      __syncthreads();
      block_compact(n_m, [](int q) { return q; }, is_member,
                    p.dbg_lib + p.targets[u.tgt_off + t].lib_dbg_off, (uint32_t)L, s_warp);
    }
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
    const size_t smem = (size_t)((max_nm + 7) / 8 * 8) * sizeof(uint32_t);  // whole blocks
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
