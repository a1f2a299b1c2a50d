// Query order: a spatially coherent ordering of the manifold points of one
// (library variable, E, tau), so that the query tiles of the fused kernel --
// consecutive runs of this order -- hold nearby points.  Nearby queries pass
// the running top-(E+2) thresholds on many of the same library points, so a
// warp takes the rare insertion path far less often than with queries in time
// order.  The order changes which tile a query belongs to and nothing else:
// every query's neighbours and prediction are the same in any order.
//
// Key: Morton interleave of the first min(E, 3) coordinates, each quantised to
// 30/D bits over the series' [min, max]; ties (and the key's low half) by the
// manifold index m, so the order is a deterministic function of the series.
// One CTA per (variable, E, tau) sorts the 64-bit keys with a bitonic network
// in shared memory when N_m <= kOrderMaxSort; a longer manifold is sorted by
// one CTA too: runs of kOrderMaxSort keys sorted in shared memory, then merged
// pairwise in global scratch (merge path: every thread finds its output range
// by a binary search on the diagonal), which gives the same order.
#include <float.h>
#include <stdint.h>

#include "ccm_internal.h"

namespace ccm {
namespace {

constexpr int kOrderThreads = 1024;

__device__ __forceinline__ uint32_t spread3(uint32_t x) {  // 10 bits -> every 3rd bit
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}
__device__ __forceinline__ uint32_t spread2(uint32_t x) {  // 15 bits -> every 2nd bit
  x &= 0x7fffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

__device__ __forceinline__ uint32_t quantise(float c, float lo, float inv, int bits) {
  const float u = (c - lo) * inv;  // in [0, 1] up to rounding
  const float top = (float)((1u << bits) - 1u);
  float v = floorf(u * (float)(1u << bits));
  v = fminf(fmaxf(v, 0.f), top);
  return (uint32_t)v;
}

// Series range of job jb (block-wide min/max).
__device__ void series_range(const float* s, int64_t n, float* lo_out, float* hi_out) {
  __shared__ float s_lo[32], s_hi[32];
  float lo = FLT_MAX, hi = -FLT_MAX;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    lo = fminf(lo, s[t]);
    hi = fmaxf(hi, s[t]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_lo[threadIdx.x >> 5] = lo;
    s_hi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  lo = s_lo[0];
  hi = s_hi[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    lo = fminf(lo, s_lo[w]);
    hi = fmaxf(hi, s_hi[w]);
  }
  __syncthreads();
  *lo_out = lo;
  *hi_out = hi;
}

// Sort key of manifold point q: (Morton code << 32) | q.
__device__ __forceinline__ unsigned long long morton_key(const float* s, int off, int tau, int E,
                                                         float lo, float inv, int q) {
  const int t = q + off;
  const int D = min(E, 3);
  uint32_t code;
  if (D == 1) {
    code = quantise(s[t], lo, inv, 30);
  } else if (D == 2) {
    code = (spread2(quantise(s[t], lo, inv, 15)) << 1) | spread2(quantise(s[t - tau], lo, inv, 15));
  } else {
    code = (spread3(quantise(s[t], lo, inv, 10)) << 2) |
           (spread3(quantise(s[t - tau], lo, inv, 10)) << 1) |
           spread3(quantise(s[t - 2 * tau], lo, inv, 10));
  }
  return ((unsigned long long)code << 32) | (unsigned)q;
}

// Ascending bitonic sort of n2 (a power of two) keys in shared memory.
__device__ void bitonic_sort(unsigned long long* k, int n2) {
  for (int size = 2; size <= n2; size <<= 1) {
    for (int jj = size >> 1; jj > 0; jj >>= 1) {
      for (int q = threadIdx.x; q < n2; q += blockDim.x) {
        const int p = q ^ jj;
        if (p > q) {
          const unsigned long long a = k[q], b = k[p];
          const bool up = (q & size) == 0;
          if ((a > b) == up) {
            k[q] = b;
            k[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kOrderThreads)
order_kernel(const float* series, const OrderJob* jobs, int32_t* order,
             unsigned long long* scratch) {
  extern __shared__ unsigned long long s_key[];
  const OrderJob jb = jobs[blockIdx.x];
  const float* s = series + jb.series_off + (int64_t)jb.j * jb.n;
  const int n_m = jb.n_m, E = jb.E, tau = jb.tau, off = (E - 1) * tau;
  int32_t* out = order + jb.order_off;
  if (n_m > kOrderMaxSort && jb.scratch_off < 0) {  // no scratch: time order
    for (int m = threadIdx.x; m < n_m; m += blockDim.x) out[m] = m;
    return;
  }
  float lo, hi;
  series_range(s, jb.n, &lo, &hi);
  const float inv = (hi > lo) ? 1.f / (hi - lo) : 0.f;
  if (n_m <= kOrderMaxSort) {
    int n2 = 1;
    while (n2 < n_m) n2 <<= 1;
    for (int q = threadIdx.x; q < n2; q += blockDim.x)
      s_key[q] = (q < n_m) ? morton_key(s, off, tau, E, lo, inv, q) : ~0ull;
    __syncthreads();
    bitonic_sort(s_key, n2);
    for (int q = threadIdx.x; q < n_m; q += blockDim.x) out[q] = (int32_t)(s_key[q] & 0xffffffffu);
    return;
  }
  // Long manifold: sorted runs of kOrderMaxSort keys, then pairwise merges.
  unsigned long long* buf[2] = {scratch + jb.scratch_off, scratch + jb.scratch_off + n_m};
  for (int r0 = 0; r0 < n_m; r0 += kOrderMaxSort) {
    const int len = min(kOrderMaxSort, n_m - r0);
    for (int q = threadIdx.x; q < kOrderMaxSort; q += blockDim.x)
      s_key[q] = (q < len) ? morton_key(s, off, tau, E, lo, inv, r0 + q) : ~0ull;
    __syncthreads();
    bitonic_sort(s_key, kOrderMaxSort);
    for (int q = threadIdx.x; q < len; q += blockDim.x) buf[0][r0 + q] = s_key[q];
    __syncthreads();
  }
  int src = 0;
  for (int width = kOrderMaxSort; width < n_m; width <<= 1, src ^= 1) {
    const unsigned long long* in = buf[src];
    unsigned long long* dst = buf[src ^ 1];
    for (int b0 = 0; b0 < n_m; b0 += 2 * width) {
      const int a_len = min(width, n_m - b0);
      const int b_len = max(0, min(width, n_m - b0 - width));
      const unsigned long long* A = in + b0;
      const unsigned long long* B = in + b0 + a_len;
      const int total = a_len + b_len;
      const int per = (total + blockDim.x - 1) / blockDim.x;
      const int k0 = min(total, (int)threadIdx.x * per), k1 = min(total, k0 + per);
      if (k0 < k1) {
        // merge path: i keys from A and k0 - i from B precede output k0 (keys are distinct)
        int lo_i = max(0, k0 - b_len), hi_i = min(k0, a_len);
        while (lo_i < hi_i) {
          const int mid = (lo_i + hi_i) >> 1;
          if (A[mid] < B[k0 - 1 - mid]) lo_i = mid + 1;
          else hi_i = mid;
        }
        int i = lo_i, jv = k0 - lo_i;
        for (int k = k0; k < k1; ++k) {
          const bool take_a = jv >= b_len || (i < a_len && A[i] < B[jv]);
          dst[b0 + k] = take_a ? A[i++] : B[jv++];
        }
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < n_m; q += blockDim.x) out[q] = (int32_t)(buf[src][q] & 0xffffffffu);
}

}  // namespace

cudaError_t order_prepare() {
  return cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kOrderMaxSort * sizeof(unsigned long long)));
}

cudaError_t launch_order(const float* series, const OrderJob* jobs, int64_t n_jobs, int max_nm,
                         int32_t* order, unsigned long long* scratch, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  int n2 = 1;
  while (n2 < max_nm && n2 < kOrderMaxSort) n2 <<= 1;
  const size_t smem = (size_t)n2 * sizeof(unsigned long long);
  order_kernel<<<(unsigned)n_jobs, kOrderThreads, smem, s>>>(series, jobs, order, scratch);
  return cudaGetLastError();
}

}  // namespace ccm
