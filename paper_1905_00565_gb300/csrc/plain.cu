// Plain GPU CCM: the straightforward CUDA form of one realization, kept as
// the comparator the batched path is measured against.  Per realization
// (pair, E, tau, L, k) it launches the sampler, a naive kNN kernel (one
// thread per query, library coordinates gathered from global memory for
// every query, a sorted insertion into a local top-(E+2) list) that writes
// the predictions, and a one-CTA FP64 Pearson kernel.  Same selection rule and
// rounding sequence as the fused kernel, hence the same neighbours.
#include <limits.h>
#include <math.h>

#include "ccm_internal.h"

namespace ccm {
namespace {

constexpr int kPlainThreads = 128;
constexpr int kRhoThreads = 1024;

__global__ void __launch_bounds__(kPlainThreads)
plain_knn_kernel(const float* series, const UnitDesc* unit, const TargetDesc* target,
                 const int32_t* lib, float* xhat) {
  const UnitDesc u = *unit;
  const TargetDesc tg = *target;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= u.n_m) return;
  const int E = u.E, tau = u.tau, off = (E - 1) * tau, K = E + 2;
  const float* sj = series + u.series_off + (int64_t)u.j * u.n;
  const float* si = series + u.series_off + (int64_t)tg.i * u.n;
  const int32_t* ul = lib + u.lib_off;
  float q[kMaxE];
  for (int e = 0; e < E; ++e) q[e] = sj[m + off - e * tau];
  float kd[kMaxE + 2];
  int kl[kMaxE + 2];
  for (int s = 0; s < K; ++s) {
    kd[s] = INFINITY;
    kl[s] = INT_MAX;
  }
  for (int a = 0; a < u.L; ++a) {
    const int l = ul[a];
    if (abs(l - m) <= u.theiler) continue;  // exclusion window (W = 0: m itself)
    float diff = __fsub_rn(q[0], sj[l + off]);
    float acc = __fmul_rn(diff, diff);
    for (int e = 1; e < E; ++e) {
      diff = __fsub_rn(q[e], sj[l + off - e * tau]);
      acc = __fmaf_rn(diff, diff, acc);
    }
    // (distance, index) order: the library may be listed in any order
    if (acc < kd[K - 1] || (acc == kd[K - 1] && l < kl[K - 1])) {
      int s = K - 1;
      while (s > 0 && (acc < kd[s - 1] || (acc == kd[s - 1] && l < kl[s - 1]))) {
        kd[s] = kd[s - 1];
        kl[s] = kl[s - 1];
        --s;
      }
      kd[s] = acc;
      kl[s] = l;
    }
  }
  // simplex projection over the E+1 nearest (the query was never a candidate)
  const float d1 = sqrt_hw(kd[0]);
  const float inv_d1 = (d1 > 0.f) ? rcp_hw(d1) : 0.f;
  float usum = 0.f, accx = 0.f;
  for (int s = 0; s <= E; ++s) {
    const float ui = simplex_u(kd[s], d1, inv_d1, u.wfloor);
    usum = __fadd_rn(usum, ui);
    const int nbc = min(max(kl[s], 0), u.n_m - 1);  // in bounds even for non-finite input
    accx = __fmaf_rn(ui, si[nbc + off], accx);
  }
  xhat[m] = __fmul_rn(accx, rcp_hw(usum));
}

__global__ void __launch_bounds__(kRhoThreads)
plain_rho_kernel(const float* series, const UnitDesc* unit, const TargetDesc* target,
                 const float* xhat, double* rho) {
  __shared__ double s_a[kRhoThreads], s_b[kRhoThreads], s_c[kRhoThreads];
  const UnitDesc u = *unit;
  const TargetDesc tg = *target;
  const int off = (u.E - 1) * u.tau;
  const float* si = series + u.series_off + (int64_t)tg.i * u.n;
  double a = 0.0, b = 0.0;
  for (int m = threadIdx.x; m < u.n_m; m += blockDim.x) {
    a += (double)si[m + off];
    b += (double)xhat[m];
  }
  s_a[threadIdx.x] = a;
  s_b[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_a[threadIdx.x] += s_a[threadIdx.x + w];
      s_b[threadIdx.x] += s_b[threadIdx.x + w];
    }
    __syncthreads();
  }
  const double mx = s_a[0] / u.n_m, my = s_b[0] / u.n_m;
  __syncthreads();
  double xx = 0.0, yy = 0.0, xy = 0.0;
  for (int m = threadIdx.x; m < u.n_m; m += blockDim.x) {
    const double x = (double)si[m + off] - mx, y = (double)xhat[m] - my;
    xx += x * x;
    yy += y * y;
    xy += x * y;
  }
  s_a[threadIdx.x] = xx;
  s_b[threadIdx.x] = yy;
  s_c[threadIdx.x] = xy;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_a[threadIdx.x] += s_a[threadIdx.x + w];
      s_b[threadIdx.x] += s_b[threadIdx.x + w];
      s_c[threadIdx.x] += s_c[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    rho[tg.out_idx] = (s_a[0] > 0.0 && s_b[0] > 0.0) ? s_c[0] / sqrt(s_a[0] * s_b[0]) : nan("");
}

}  // namespace

cudaError_t launch_plain_unit(const float* series, const UnitDesc* unit_dev, const UnitDesc& unit,
                              const TargetDesc* target_dev, const int32_t* lib,
                              float* xhat_scratch, double* rho_out, cudaStream_t s) {
  const unsigned grid = (unsigned)((unit.n_m + kPlainThreads - 1) / kPlainThreads);
  plain_knn_kernel<<<grid, kPlainThreads, 0, s>>>(series, unit_dev, target_dev, lib, xhat_scratch);
  plain_rho_kernel<<<1, kRhoThreads, 0, s>>>(series, unit_dev, target_dev, xhat_scratch, rho_out);
  return cudaGetLastError();
}

}  // namespace ccm
