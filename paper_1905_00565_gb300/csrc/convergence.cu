// Convergence decision on the rho grid (paper Sect. 1: cross-map skill should
// rise with the library size L, judged over the r realizations; the paper
// states no test, the one used here is a one-sided Jonckheere-Terpstra trend
// test over the L groups).
//
// One CTA per (pair, E, tau) row of rho [rows][n_L][r]: the row is staged in
// shared memory with the L groups in increasing L and every group is sorted;
// then each finite member y adds, for every earlier group, twice the number of
// its members below y and once those equal to y (two binary searches), so 2J
// is an exact integer.  Non-finite rho (a realization with zero variance) are
// left out.  Thread 0 forms E[J], Var[J] (no tie correction), z and the group
// means (summed before sorting, in realization order) with explicit
// round-to-nearest operations in a fixed order: group sizes summed in
// increasing L, then E[J], Var[J] and z, so the result depends on nothing but
// the row.
#include <math.h>
#include <stdint.h>

#include "ccm_internal.h"

namespace ccm {
namespace {

constexpr int kConvThreads = 256;

// Ascending sort, by the whole block, of each of n_g groups of n doubles
// (group g at v + g*n): a bitonic network whose comparators all put the
// smaller value at the lower index (the first step of every merge compares
// mirrored positions), over the next power of two with virtual +infinity
// beyond n, so positions at or above n never take part.  One barrier per step.
__device__ void block_sort_groups(double* v, int n_g, int n) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  const int half = n2 / 2, pairs = n_g * half;
  for (int k = 2; k <= n2; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < pairs; t += blockDim.x) {
        const int g = t / half, tp = t - g * half;
        // pair tp of this step: block of size 2*jj, offset inside the half
        const int blk = tp / jj, off = tp - blk * jj;
        const int i = blk * 2 * jj + off;
        const int j = (jj == (k >> 1)) ? (blk * 2 * jj + 2 * jj - 1 - off) : (i + jj);
        if (j < n) {
          double* w = v + g * n;
          const double a = w[i], c = w[j];
          if (c < a) {
            w[i] = c;
            w[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

// First position in v[0..n) (ascending) whose value is not below x / above x.
__device__ __forceinline__ int lower_pos(const double* v, int n, double x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int upper_pos(const double* v, int n, double x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kConvThreads)
convergence_kernel(const double* rho, int32_t n_L, int32_t r, ConvOrder ord, double z_crit,
                   ConvergenceRow* out) {
  extern __shared__ double s_val[];           // [n_L][r], groups in increasing L
  __shared__ unsigned long long s_j2[kConvThreads / 32];
  __shared__ int s_cnt[kMaxConvGroups];
  __shared__ double s_mean[2];
  const int tid = threadIdx.x;
  const int64_t row = blockIdx.x;
  const int T = n_L * r;
  const double* src = rho + row * (int64_t)T;
  for (int g = tid; g < n_L; g += kConvThreads) s_cnt[g] = 0;
  __syncthreads();
  for (int i = tid; i < T; i += kConvThreads) {
    const int g = i / r, k = i - g * r;
    const double v = src[(int64_t)ord.group[g] * r + k];
    const bool fin = isfinite(v);
    s_val[i] = fin ? v : INFINITY;  // non-finite realizations sort last and are not counted
    if (fin) atomicAdd(&s_cnt[g], 1);
  }
  __syncthreads();
  // group means of the finite realizations, summed in realization order (before sorting)
  if (tid < 2) {
    const int g = (tid == 0) ? 0 : n_L - 1;
    double t = 0.0;
    for (int k = 0; k < r; ++k) {
      const double v = s_val[g * r + k];
      if (v != INFINITY) t = __dadd_rn(t, v);
    }
    s_mean[tid] = (s_cnt[g] > 0) ? __ddiv_rn(t, (double)s_cnt[g]) : nan("");
  }
  __syncthreads();
  block_sort_groups(s_val, n_L, r);
  // 2J: for each finite y, the members of earlier groups below it (2 each) and
  // equal to it (1 each), by binary searches in the sorted groups
  unsigned long long j2 = 0ull;
  for (int i = tid; i < T; i += kConvThreads) {
    const int g = i / r;
    const double y = s_val[i];
    if (i - g * r >= s_cnt[g]) continue;  // a non-finite realization
    for (int h = 0; h < g; ++h) {
      const double* v = s_val + h * r;
      const int lo = lower_pos(v, s_cnt[h], y), hi = upper_pos(v, s_cnt[h], y);
      j2 += 2ull * (unsigned long long)lo + (unsigned long long)(hi - lo);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) j2 += __shfl_xor_sync(0xffffffffu, j2, o);
  if ((tid & 31) == 0) s_j2[tid >> 5] = j2;
  __syncthreads();
  if (tid != 0) return;
  unsigned long long J2 = 0ull;
  for (int w = 0; w < kConvThreads / 32; ++w) J2 += s_j2[w];
  double N = 0.0, S2 = 0.0, S3 = 0.0;
  for (int g = 0; g < n_L; ++g) {
    const double n = (double)s_cnt[g];
    N = __dadd_rn(N, n);
    S2 = __dadd_rn(S2, __dmul_rn(n, n));
    S3 = __dadd_rn(S3, __dmul_rn(__dmul_rn(n, n), __dadd_rn(__dmul_rn(2.0, n), 3.0)));
  }
  const double J = 0.5 * (double)J2;  // exact: J2 < 2^53
  const double mean = __ddiv_rn(__dsub_rn(__dmul_rn(N, N), S2), 4.0);
  const double var = __ddiv_rn(
      __dsub_rn(__dmul_rn(__dmul_rn(N, N), __dadd_rn(__dmul_rn(2.0, N), 3.0)), S3), 72.0);
  ConvergenceRow o;
  o.jt = J;
  o.z = (var > 0.0) ? __ddiv_rn(__dsub_rn(J, mean), __dsqrt_rn(var)) : nan("");
  o.rho_first = s_mean[0];
  o.rho_last = s_mean[1];
  o.n_valid = (int32_t)N;
  o.converged = (o.z > z_crit && o.rho_last > o.rho_first && o.rho_last > 0.0) ? 1 : 0;
  out[row] = o;
}

}  // namespace

size_t convergence_smem(int32_t n_L, int32_t r) { return (size_t)n_L * (size_t)r * 8; }

cudaError_t convergence_prepare() {
  return cudaFuncSetAttribute(convergence_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kMaxConvValues * 8));
}

cudaError_t launch_convergence(const double* rho, int64_t n_rows, int32_t n_L, int32_t r,
                               const ConvOrder& ord, double z_crit, ConvergenceRow* out,
                               cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  convergence_kernel<<<(unsigned)n_rows, kConvThreads, convergence_smem(n_L, r), s>>>(
      rho, n_L, r, ord, z_crit, out);
  return cudaGetLastError();
}

}  // namespace ccm
