// CPU oracle for convergent cross mapping (CCM) -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of what the GPU path computes,
// used by the tests, by the smoke check and by the benchmark's CPU baseline.
// It shares no code, header, table or constant with the CUDA library; the
// product path never calls it.
//
// What it computes (paper Sect. 1, Sect. 2.1, Sect. 3.1, Sect. 3.2 and the
// method's source, Sugihara et al. 2012, which the paper cites for CCM):
//   * shadow manifold of library variable j with embedding dimension E and
//     delay tau: M_j(m) = (s_j[t], s_j[t-tau], ..., s_j[t-(E-1)tau]) with
//     t = m + (E-1)tau, m in [0, N_m), N_m = N - (E-1)tau;
//   * r random libraries of L manifold points drawn without replacement
//     (Sect. 1, Sect. 3.1), here by random-key selection with Philox4x64-10;
//   * for every manifold point its E+1 nearest library neighbours, itself
//     excluded (Sect. 3.2: "the E+1 nearest neighbors");
//   * simplex projection (Sect. 2.1): u_i = exp(-d_i/d_1), w_i = u_i / sum u,
//     Xhat(t) = sum w_i X(t_i);
//   * skill = Pearson correlation of X and Xhat (Sect. 2.1).
// Two options that the paper does not discuss but common CCM implementations
// carry, both off by default (the paper's method):
//   * an exclusion (Theiler) window W >= 0: a library point l is a neighbour
//     candidate of query m only when |l - m| > W (W = 0: only m itself is
//     excluded, the paper's rule), so that points close in time do not
//     predict each other;
//   * a weight floor f >= 0: u_i = max(exp(-d_i/d_1), f) before the
//     normalisation, so that a far neighbour keeps a small positive weight.
//
// Precision: the neighbour selection can be taken on FP32 squared distances
// accumulated in coordinate order with one rounding per fused multiply-add
// (the precision the GPU kernel decides in), or on FP64 squared distances.
// Distances used in the weights, the weights, Xhat and rho are FP64.
//
// Parity pins live in tests/test_oracle_*.py: Philox against numpy's
// Philox4x64-10, neighbours against brute force on tiny inputs, a hand-worked
// 10-point simplex example, rho against numpy.corrcoef, invariances, and the
// known convergence of the coupled logistic map.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (see build.py);
// -ffp-contract=off keeps every FP64 sum an ordinary add, so that pure-Python
// brute force in the tests reproduces it bit for bit.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Philox4x64-10 counter-based generator, restated from its published
// definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications with the
// round keys bumped by two Weyl constants between rounds.
// ---------------------------------------------------------------------------
const uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ULL;
const uint64_t kPhiloxM1 = 0xCA5A826395121157ULL;
const uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ULL;  // golden ratio
const uint64_t kPhiloxW1 = 0xBB67AE8584CAA73BULL;  // sqrt(3) - 1

void mul_hi_lo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void philox4x64_10(const uint64_t in_ctr[4], const uint64_t in_key[2], uint64_t out[4]) {
  uint64_t c0 = in_ctr[0], c1 = in_ctr[1], c2 = in_ctr[2], c3 = in_ctr[3];
  uint64_t k0 = in_key[0], k1 = in_key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul_hi_lo(kPhiloxM0, c0, &hi0, &lo0);
    mul_hi_lo(kPhiloxM1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ---------------------------------------------------------------------------
// Library sampling without replacement (Sect. 1: r random subsamples of size
// L; Sect. 3.1; the paper names no generator).  Random-key selection:
// manifold point m gets the key whose high 32 bits are 32-bit half number
// m mod 8 of the Philox block at counter (floor(m/8), k, L,
// (j<<16)|(E<<8)|tau) under key (seed, 0) -- the halves taken in the order
// high(w0), low(w0), high(w1), ..., low(w3) -- and whose low 32 bits are m.
// The L points with the smallest keys form the library, listed in ascending
// m.  Keys are distinct (m is in them), so the choice has no ties.
// ---------------------------------------------------------------------------
void sample_library(int64_t n_m, int64_t L, int32_t j, int32_t E, int32_t tau, int32_t k,
                    uint64_t seed, int32_t* lib) {
  std::vector<uint64_t> keys((size_t)n_m);
  const uint64_t key[2] = {seed, 0};
  for (int64_t m = 0; m < n_m; ++m) {
    const uint64_t ctr[4] = {(uint64_t)(m / 8), (uint64_t)k, (uint64_t)L,
                             ((uint64_t)j << 16) | ((uint64_t)E << 8) | (uint64_t)tau};
    uint64_t w[4];
    philox4x64_10(ctr, key, w);
    const uint64_t word = w[(m % 8) / 2];
    const uint64_t half = (m % 2 == 0) ? (word >> 32) : (word & 0xFFFFFFFFULL);
    keys[(size_t)m] = (half << 32) | (uint64_t)m;
  }
  std::sort(keys.begin(), keys.end());
  std::vector<int32_t> chosen((size_t)L);
  for (int64_t q = 0; q < L; ++q) chosen[(size_t)q] = (int32_t)(keys[(size_t)q] & 0xFFFFFFFFULL);
  std::sort(chosen.begin(), chosen.end());
  for (int64_t q = 0; q < L; ++q) lib[q] = chosen[(size_t)q];
}

// Coordinate e of manifold point m: s[m + (E-1)tau - e tau].
inline float coord(const float* s, int32_t E, int32_t tau, int64_t m, int32_t e) {
  return s[m + (int64_t)(E - 1) * tau - (int64_t)e * tau];
}

// FP32 squared distance, accumulated in coordinate order: the first term is a
// rounded product, every later term one fused multiply-add (fmaf rounds once).
float sqdist_fp32(const float* s, int32_t E, int32_t tau, int64_t a, int64_t b) {
  float diff = coord(s, E, tau, a, 0) - coord(s, E, tau, b, 0);
  float acc = diff * diff;
  for (int32_t e = 1; e < E; ++e) {
    diff = coord(s, E, tau, a, e) - coord(s, E, tau, b, e);
    acc = std::fmaf(diff, diff, acc);
  }
  return acc;
}

// FP64 squared distance of the FP32 coordinates promoted to FP64.
double sqdist_fp64(const float* s, int32_t E, int32_t tau, int64_t a, int64_t b) {
  double acc = 0.0;
  for (int32_t e = 0; e < E; ++e) {
    double diff = (double)coord(s, E, tau, a, e) - (double)coord(s, E, tau, b, e);
    acc = acc + diff * diff;
  }
  return acc;
}

// ---------------------------------------------------------------------------
// E+1 nearest library neighbours of every manifold point, itself excluded
// (Sect. 3.2).  All library distances are computed and ordered by
// (squared distance, manifold index); the first E+1 are kept.  Squared
// distance orders like distance.  Exclusion is by index: another point at
// distance 0 stays eligible.
// ---------------------------------------------------------------------------
void query_neighbours(const float* s, int32_t E, int32_t tau, const int32_t* lib, int64_t L,
                      int32_t select_fp64, int32_t theiler, int64_t m,
                      std::vector<std::pair<double, int32_t>>* cand, int32_t* nbr_row) {
  const int32_t kk = E + 1;
  cand->clear();
  for (int64_t q = 0; q < L; ++q) {
    const int32_t l = lib[q];
    if (std::llabs((long long)l - (long long)m) <= theiler) continue;  // m itself when W = 0
    const double d2 = select_fp64 ? sqdist_fp64(s, E, tau, m, l)
                                  : (double)sqdist_fp32(s, E, tau, m, l);
    cand->push_back(std::make_pair(d2, l));
  }
  std::partial_sort(cand->begin(), cand->begin() + kk, cand->end());
  for (int32_t i = 0; i < kk; ++i) nbr_row[i] = (*cand)[(size_t)i].second;
}

void neighbours(const float* s, int64_t n, int32_t E, int32_t tau, const int32_t* lib,
                int64_t L, int32_t select_fp64, int32_t theiler, int32_t* nbr) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  std::vector<std::pair<double, int32_t>> cand;
  cand.reserve((size_t)L);
  for (int64_t m = 0; m < n_m; ++m)
    query_neighbours(s, E, tau, lib, L, select_fp64, theiler, m, &cand, nbr + m * (E + 1));
}

// ---------------------------------------------------------------------------
// Simplex projection (Sect. 2.1): FP64 distances d_1 <= ... <= d_{E+1} of the
// given neighbours, u_i = exp(-d_i/d_1), w_i = u_i / sum u, Xhat = sum w_i
// x[t_i].  When d_1 = 0, u_i is the limit of exp(-d_i/d_1) as d_1 -> 0+:
// 1 for d_i = 0 and 0 otherwise.  With a weight floor f, u_i = max(u_i, f).
// ---------------------------------------------------------------------------
double query_predict(const float* lib_s, const float* tgt_s, int32_t E, int32_t tau,
                     double weight_floor, const int32_t* nbr_row, int64_t m) {
  const int32_t kk = E + 1;
  std::vector<double> d((size_t)kk), u((size_t)kk);
  for (int32_t i = 0; i < kk; ++i) d[(size_t)i] = std::sqrt(sqdist_fp64(lib_s, E, tau, m, nbr_row[i]));
  double d1 = d[0];
  for (int32_t i = 1; i < kk; ++i) d1 = std::min(d1, d[(size_t)i]);
  double usum = 0.0;
  for (int32_t i = 0; i < kk; ++i) {
    if (d1 > 0.0)
      u[(size_t)i] = std::exp(-d[(size_t)i] / d1);
    else
      u[(size_t)i] = (d[(size_t)i] == 0.0) ? 1.0 : 0.0;
    u[(size_t)i] = std::max(u[(size_t)i], weight_floor);
    usum += u[(size_t)i];
  }
  double acc = 0.0;
  for (int32_t i = 0; i < kk; ++i) {
    const int64_t t_i = nbr_row[i] + (int64_t)(E - 1) * tau;
    acc += (u[(size_t)i] / usum) * (double)tgt_s[t_i];
  }
  return acc;
}

void predict(const float* lib_s, const float* tgt_s, int64_t n, int32_t E, int32_t tau,
             double weight_floor, const int32_t* nbr, double* xhat) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  for (int64_t m = 0; m < n_m; ++m)
    xhat[m] = query_predict(lib_s, tgt_s, E, tau, weight_floor, nbr + m * (E + 1), m);
}

// Option check shared by the entry points: W >= 0 with every query keeping at
// least E+1 candidates (L >= E + 2 + 2W), and a finite floor f >= 0.
bool options_ok(int32_t E, int64_t L, int32_t theiler, double weight_floor) {
  return theiler >= 0 && L >= (int64_t)E + 2 + 2 * (int64_t)theiler &&
         std::isfinite(weight_floor) && weight_floor >= 0.0;
}

// Pearson correlation, two passes in FP64; NaN when either variance is 0.
double pearson(const double* x, const double* y, int64_t n) {
  double mx = 0.0, my = 0.0;
  for (int64_t q = 0; q < n; ++q) { mx += x[q]; my += y[q]; }
  mx /= (double)n;
  my /= (double)n;
  double sxx = 0.0, syy = 0.0, sxy = 0.0;
  for (int64_t q = 0; q < n; ++q) {
    const double a = x[q] - mx, b = y[q] - my;
    sxx += a * a;
    syy += b * b;
    sxy += a * b;
  }
  if (sxx == 0.0 || syy == 0.0) return std::nan("");
  return sxy / std::sqrt(sxx * syy);
}

// The observed target at the query times t_m = m + (E-1)tau, as FP64.
void observed(const float* tgt_s, int64_t n, int32_t E, int32_t tau, double* x) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  for (int64_t m = 0; m < n_m; ++m) x[m] = (double)tgt_s[m + (int64_t)(E - 1) * tau];
}

// ---------------------------------------------------------------------------
// Convergence decision for one (pair, E, tau) row of the rho grid (Sect. 1:
// skill should rise with L, judged over the r realizations; the paper states
// no test, so this is a chosen reading).  Groups are the L values in
// increasing order, each holding the finite rho of its realizations.  The
// Jonckheere-Terpstra statistic counts, over every pair of groups a < b and
// every pair of members (x in a, y in b), 1 when y > x and 1/2 when y == x.
// With no trend (all rho exchangeable) and N = sum n_g:
//   E[J]   = (N^2 - sum n_g^2) / 4,
//   Var[J] = (N^2 (2N + 3) - sum n_g^2 (2 n_g + 3)) / 72   (no tie correction),
//   z      = (J - E[J]) / sqrt(Var[J]).
// The row converges when z > z_crit, the mean rho at the largest L exceeds
// the mean at the smallest L, and the mean at the largest L is positive.
// ---------------------------------------------------------------------------
struct Convergence {
  double rho_first, rho_last, jt, z;
  int32_t n_valid, converged;
};

Convergence convergence_row(const double* row, int32_t n_L, const int64_t* L, int32_t r,
                            double z_crit) {
  std::vector<int32_t> order((size_t)n_L);
  for (int32_t l = 0; l < n_L; ++l) order[(size_t)l] = l;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return L[a] < L[b]; });
  std::vector<std::vector<double>> g((size_t)n_L);
  for (int32_t q = 0; q < n_L; ++q) {
    const double* x = row + (int64_t)order[(size_t)q] * r;
    for (int32_t k = 0; k < r; ++k)
      if (std::isfinite(x[k])) g[(size_t)q].push_back(x[k]);
  }
  Convergence c;
  double J = 0.0, N = 0.0, S2 = 0.0, S3 = 0.0;
  for (int32_t a = 0; a < n_L; ++a)
    for (int32_t b = a + 1; b < n_L; ++b)
      for (double x : g[(size_t)a])
        for (double y : g[(size_t)b]) J += (y > x) ? 1.0 : (y == x ? 0.5 : 0.0);
  for (int32_t a = 0; a < n_L; ++a) {
    const double n = (double)g[(size_t)a].size();
    N += n;
    S2 += n * n;
    S3 += n * n * (2.0 * n + 3.0);
  }
  const double mean = (N * N - S2) / 4.0;
  const double var = (N * N * (2.0 * N + 3.0) - S3) / 72.0;
  c.jt = J;
  c.z = var > 0.0 ? (J - mean) / std::sqrt(var) : std::nan("");
  auto avg = [](const std::vector<double>& v) {
    double t = 0.0;
    for (double x : v) t += x;
    return v.empty() ? std::nan("") : t / (double)v.size();
  };
  c.rho_first = avg(g.front());
  c.rho_last = avg(g.back());
  c.n_valid = (int32_t)N;
  c.converged = (c.z > z_crit && c.rho_last > c.rho_first && c.rho_last > 0.0) ? 1 : 0;
  return c;
}

}  // namespace

extern "C" {

void oracle_philox4x64_10(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
  philox4x64_10(ctr, key, out);
}

// Library of unit (j, E, tau, L, k): L ascending manifold indices in [0, n_m).
int oracle_library(int64_t n_m, int64_t L, int32_t j, int32_t E, int32_t tau, int32_t k,
                   uint64_t seed, int32_t* lib_out) {
  if (L < 1 || L > n_m) return -1;
  sample_library(n_m, L, j, E, tau, k, seed, lib_out);
  return 0;
}

// E+1 nearest neighbours [N_m][E+1] of every manifold point of series s.
int oracle_neighbours(const float* s, int64_t n, int32_t E, int32_t tau, const int32_t* lib,
                      int64_t L, int32_t select_fp64, int32_t theiler, int32_t* nbr_out) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  if (E < 1 || tau < 1 || n_m < 1 || L < E + 2 || L > n_m) return -1;
  if (!options_ok(E, L, theiler, 0.0)) return -1;
  neighbours(s, n, E, tau, lib, L, select_fp64, theiler, nbr_out);
  return 0;
}

// Simplex predictions [N_m] from given neighbour lists (also the "replay" of
// a neighbour set found elsewhere).
int oracle_predict(const float* lib_s, const float* tgt_s, int64_t n, int32_t E, int32_t tau,
                   double weight_floor, const int32_t* nbr, double* xhat_out) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  if (E < 1 || tau < 1 || n_m < 1) return -1;
  if (!std::isfinite(weight_floor) || weight_floor < 0.0) return -1;
  predict(lib_s, tgt_s, n, E, tau, weight_floor, nbr, xhat_out);
  return 0;
}

// Neighbours [nq][E+1] and predictions [nq] of the listed query points only
// (for checking sampled outputs of large problems).
int oracle_query_subset(const float* lib_s, const float* tgt_s, int64_t n, int32_t E, int32_t tau,
                        const int32_t* lib, int64_t L, const int64_t* queries, int64_t nq,
                        int32_t select_fp64, int32_t theiler, double weight_floor,
                        int32_t* nbr_out, double* xhat_out) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  if (E < 1 || tau < 1 || n_m < 1 || L < E + 2 || L > n_m) return -1;
  if (!options_ok(E, L, theiler, weight_floor)) return -1;
  std::vector<std::pair<double, int32_t>> cand;
  cand.reserve((size_t)L);
  for (int64_t q = 0; q < nq; ++q) {
    if (queries[q] < 0 || queries[q] >= n_m) return -1;
    query_neighbours(lib_s, E, tau, lib, L, select_fp64, theiler, queries[q], &cand,
                     nbr_out + q * (E + 1));
    xhat_out[q] = query_predict(lib_s, tgt_s, E, tau, weight_floor, nbr_out + q * (E + 1),
                                queries[q]);
  }
  return 0;
}

// How close query m's neighbour set is to a tie at its boundary: the FP64
// distances (selection in FP64) of its (E+1)-th and (E+2)-th nearest
// candidates, d_a <= d_b, give gap = (d_b - d_a) / d_b; +inf when the query
// has only E+1 candidates, 0 when d_b = 0.  A neighbour set chosen in a lower
// precision can differ from the FP64 one only where this gap is small: the
// point swapped out is no farther than d_a and the point swapped in no
// nearer than d_b in FP64, yet the two compared the other way.
int oracle_query_margin(const float* s, int64_t n, int32_t E, int32_t tau, const int32_t* lib,
                        int64_t L, const int64_t* queries, int64_t nq, int32_t theiler,
                        double* gap_out) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  if (E < 1 || tau < 1 || n_m < 1 || L < E + 2 || L > n_m) return -1;
  if (!options_ok(E, L, theiler, 0.0)) return -1;
  std::vector<double> d2;
  d2.reserve((size_t)L);
  for (int64_t q = 0; q < nq; ++q) {
    const int64_t m = queries[q];
    if (m < 0 || m >= n_m) return -1;
    d2.clear();
    for (int64_t a = 0; a < L; ++a) {
      const int32_t l = lib[a];
      if (std::llabs((long long)l - (long long)m) <= theiler) continue;
      d2.push_back(sqdist_fp64(s, E, tau, m, l));
    }
    if ((int64_t)d2.size() < E + 2) {
      gap_out[q] = INFINITY;
      continue;
    }
    std::partial_sort(d2.begin(), d2.begin() + (E + 2), d2.end());
    const double da = std::sqrt(d2[(size_t)E]), db = std::sqrt(d2[(size_t)E + 1]);
    gap_out[q] = (db > 0.0) ? (db - da) / db : 0.0;
  }
  return 0;
}

double oracle_pearson(const double* x, const double* y, int64_t n) { return pearson(x, y, n); }

// Pearson rho of observed target vs predictions given as FP64 [N_m].
double oracle_skill(const float* tgt_s, int64_t n, int32_t E, int32_t tau, const double* xhat) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  std::vector<double> x((size_t)n_m);
  observed(tgt_s, n, E, tau, x.data());
  return pearson(x.data(), xhat, n_m);
}

// One unit (pair (j, i), E, tau, L, realization k).  Optional outputs:
// library [L], neighbours [N_m][E+1], predictions [N_m] (pass NULL to skip).
int oracle_ccm_unit(const float* series, int32_t V, int64_t n, int32_t j, int32_t i, int32_t E,
                    int32_t tau, int64_t L, int32_t k, uint64_t seed, int32_t select_fp64,
                    int32_t theiler, double weight_floor, double* rho_out, int32_t* lib_out,
                    int32_t* nbr_out, double* xhat_out) {
  const int64_t n_m = n - (int64_t)(E - 1) * tau;
  if (j < 0 || j >= V || i < 0 || i >= V || i == j) return -1;
  if (E < 1 || E > 10 || tau < 1 || n_m < 1 || L < E + 2 || L > n_m || k < 0) return -1;
  if (!options_ok(E, L, theiler, weight_floor)) return -1;
  const float* s_j = series + (int64_t)j * n;
  const float* s_i = series + (int64_t)i * n;
  std::vector<int32_t> lib((size_t)L), nbr((size_t)(n_m * (E + 1)));
  std::vector<double> xhat((size_t)n_m);
  sample_library(n_m, L, j, E, tau, k, seed, lib.data());
  neighbours(s_j, n, E, tau, lib.data(), L, select_fp64, theiler, nbr.data());
  predict(s_j, s_i, n, E, tau, weight_floor, nbr.data(), xhat.data());
  std::vector<double> x((size_t)n_m);
  observed(s_i, n, E, tau, x.data());
  *rho_out = pearson(x.data(), xhat.data(), n_m);
  if (lib_out) std::memcpy(lib_out, lib.data(), sizeof(int32_t) * (size_t)L);
  if (nbr_out) std::memcpy(nbr_out, nbr.data(), sizeof(int32_t) * nbr.size());
  if (xhat_out) std::memcpy(xhat_out, xhat.data(), sizeof(double) * (size_t)n_m);
  return 0;
}

// A whole sweep: rho[pair][E][tau][L][k], plain nested loops.
int oracle_ccm(const float* series, int32_t V, int64_t n, const int32_t* pairs, int32_t n_pairs,
               const int32_t* Es, int32_t n_E, const int32_t* taus, int32_t n_tau,
               const int64_t* Ls, int32_t n_L, int32_t r, uint64_t seed, int32_t select_fp64,
               int32_t theiler, double weight_floor, double* rho_out) {
  int64_t o = 0;
  for (int32_t p = 0; p < n_pairs; ++p)
    for (int32_t e = 0; e < n_E; ++e)
      for (int32_t t = 0; t < n_tau; ++t)
        for (int32_t l = 0; l < n_L; ++l)
          for (int32_t k = 0; k < r; ++k) {
            const int rc = oracle_ccm_unit(series, V, n, pairs[2 * p], pairs[2 * p + 1], Es[e],
                                           taus[t], Ls[l], k, seed, select_fp64, theiler,
                                           weight_floor, &rho_out[o], nullptr, nullptr, nullptr);
            if (rc != 0) return rc;
            ++o;
          }
  return 0;
}

// Convergence decision for every (pair, E, tau) row of rho [rows][n_L][r]:
// out[row*6 .. row*6+5] = rho_first, rho_last, J, z, n_valid, converged.
int oracle_convergence(const double* rho, int64_t n_rows, int32_t n_L, const int64_t* L,
                       int32_t r, double z_crit, double* out) {
  if (n_rows < 0 || n_L < 2 || r < 1) return -1;
  for (int64_t q = 0; q < n_rows; ++q) {
    const Convergence c = convergence_row(rho + q * (int64_t)n_L * r, n_L, L, r, z_crit);
    double* o = out + 6 * q;
    o[0] = c.rho_first;
    o[1] = c.rho_last;
    o[2] = c.jt;
    o[3] = c.z;
    o[4] = (double)c.n_valid;
    o[5] = (double)c.converged;
  }
  return 0;
}

}  // extern "C"
