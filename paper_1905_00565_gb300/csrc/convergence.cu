// Convergence decision on the rho grid (paper Sect. 1: cross-map skill should
// rise with the library size L, judged over the r realizations; the paper
// states no test, the one used here is a one-sided Jonckheere-Terpstra trend
// test over the L groups).
//
// One CTA per (pair, E, tau) row of rho [rows][n_L][r]: the row is staged in
// shared memory with the L groups in increasing L, every thread counts, for
// its members x, the members y of later groups with y > x (2) or y == x (1),
// so 2J is an exact integer; NaN (a realization with zero variance) compares
// false both ways and is left out of the counts.  Thread 0 forms E[J],
// Var[J] (no tie correction), z and the group means with explicit
// round-to-nearest operations in a fixed order.
#include <math.h>
#include <stdint.h>

#include "ccm_internal.h"

namespace ccm {
namespace {

constexpr int kConvThreads = 256;

__global__ void __launch_bounds__(kConvThreads)
convergence_kernel(const double* rho, int32_t n_L, int32_t r, ConvOrder ord, double z_crit,
                   ConvergenceRow* out) {
  extern __shared__ double s_val[];           // [n_L][r], groups in increasing L
  __shared__ unsigned long long s_j2[kConvThreads / 32];
  __shared__ int s_cnt[kMaxConvGroups];
  const int tid = threadIdx.x;
  const int64_t row = blockIdx.x;
  const int T = n_L * r;
  const double* src = rho + row * (int64_t)T;
  for (int g = tid; g < n_L; g += kConvThreads) s_cnt[g] = 0;
  for (int i = tid; i < T; i += kConvThreads) {
    const int g = i / r, k = i - g * r;
    const double v = src[(int64_t)ord.group[g] * r + k];
    s_val[i] = isfinite(v) ? v : nan("");  // NaN compares false both ways
  }
  __syncthreads();
  unsigned long long j2 = 0ull;
  for (int a = tid; a < T; a += kConvThreads) {
    const double x = s_val[a];
    if (isfinite(x)) atomicAdd(&s_cnt[a / r], 1);
    for (int b = (a / r + 1) * r; b < T; ++b) {
      const double y = s_val[b];
      j2 += (y > x) ? 2ull : ((y == x) ? 1ull : 0ull);
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
  // group means of the finite realizations, summed in realization order
  double m[2];
  for (int e = 0; e < 2; ++e) {
    const int g = (e == 0) ? 0 : n_L - 1;
    double t = 0.0;
    for (int k = 0; k < r; ++k) {
      const double v = s_val[g * r + k];
      if (isfinite(v)) t = __dadd_rn(t, v);
    }
    m[e] = (s_cnt[g] > 0) ? __ddiv_rn(t, (double)s_cnt[g]) : nan("");
  }
  o.rho_first = m[0];
  o.rho_last = m[1];
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
