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
// in shared memory when N_m <= kOrderMaxSort; longer manifolds keep time order.
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

__global__ void __launch_bounds__(kOrderThreads)
order_kernel(const float* series, const OrderJob* jobs, int32_t* order) {
  extern __shared__ unsigned long long s_key[];
  __shared__ float s_lo[32], s_hi[32];
  const OrderJob jb = jobs[blockIdx.x];
  const float* s = series + jb.series_off + (int64_t)jb.j * jb.n;
  const int n_m = jb.n_m, E = jb.E, tau = jb.tau, off = (E - 1) * tau;
  int32_t* out = order + jb.order_off;
  if (n_m > kOrderMaxSort) {  // long manifold: time order
    for (int m = threadIdx.x; m < n_m; m += blockDim.x) out[m] = m;
    return;
  }
  // series range
  float lo = FLT_MAX, hi = -FLT_MAX;
  for (int64_t t = threadIdx.x; t < jb.n; t += blockDim.x) {
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
  const float inv = (hi > lo) ? 1.f / (hi - lo) : 0.f;
  const int D = min(E, 3);
  int n2 = 1;
  while (n2 < n_m) n2 <<= 1;
  for (int q = threadIdx.x; q < n2; q += blockDim.x) {
    unsigned long long key = ~0ull;
    if (q < n_m) {
      const int t = q + off;
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
      key = ((unsigned long long)code << 32) | (unsigned)q;
    }
    s_key[q] = key;
  }
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= n2; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int q = threadIdx.x; q < n2; q += blockDim.x) {
        const int p = q ^ jj;
        if (p > q) {
          const unsigned long long a = s_key[q], b = s_key[p];
          const bool up = (q & k) == 0;
          if ((a > b) == up) {
            s_key[q] = b;
            s_key[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < n_m; q += blockDim.x) out[q] = (int32_t)(s_key[q] & 0xffffffffu);
}

}  // namespace

cudaError_t order_prepare() {
  return cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kOrderMaxSort * sizeof(unsigned long long)));
}

cudaError_t launch_order(const float* series, const OrderJob* jobs, int64_t n_jobs, int max_nm,
                         int32_t* order, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  int n2 = 1;
  while (n2 < max_nm && n2 < kOrderMaxSort) n2 <<= 1;
  const size_t smem = (size_t)n2 * sizeof(unsigned long long);
  order_kernel<<<(unsigned)n_jobs, kOrderThreads, smem, s>>>(series, jobs, order);
  return cudaGetLastError();
}

}  // namespace ccm
