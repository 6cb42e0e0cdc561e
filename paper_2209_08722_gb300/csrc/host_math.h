// Host-side numerical helpers of the solver (plain C++, no CUDA): the extreme
// Ritz values behind the Chebyshev interval (Section 3.2) and the check of a
// sketch draw (Lemma 4.1).  Kept free of CUDA so that they can be compiled
// and tested on their own.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace lpk {

// Smallest and largest eigenvalue of the symmetric tridiagonal matrix with
// diagonal dg (k entries) and off-diagonal off (k - 1 entries), by bisection
// on Sturm sequence counts (the number of negative pivots of T - x I equals
// the number of eigenvalues below x), inside the Gershgorin interval.
inline void tridiag_extremes(const std::vector<double>& dg, const std::vector<double>& off, double* lo,
                             double* hi) {
  const int k = (int)dg.size();
  double gl = 1e300, gu = -1e300;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(off[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(off[i]) : 0.0);
    gl = std::min(gl, dg[i] - r);
    gu = std::max(gu, dg[i] + r);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
      const double o2 = i > 0 ? off[i - 1] * off[i - 1] : 0.0;
      q = dg[i] - x - (i > 0 ? o2 / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  auto kth = [&](int idx) {  // idx-th smallest eigenvalue (0-based)
    double a = gl, b = gu;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (count_below(mid) > idx) b = mid;
      else a = mid;
    }
    return 0.5 * (a + b);
  };
  *lo = kth(0);
  *hi = kth(k - 1);
}

// Extreme Ritz values of the preconditioned operator from the first kk CG
// steps: the Lanczos tridiagonal that CG's coefficients define has diagonal
// 1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal sqrt(beta_j)/alpha_j,
// with alpha_j at coef[2j] and beta_j at coef[2j+1].  Returns false (and
// leaves lo, hi alone) when the recurrence has broken down (a non-positive
// alpha or a negative beta).
inline bool lanczos_extremes(const double* coef, int kk, double* lo, double* hi) {
  if (kk <= 0) return false;
  std::vector<double> dg(kk), off(std::max(0, kk - 1));
  for (int j = 0; j < kk; ++j) {
    const double al = coef[2 * j], be_prev = j > 0 ? coef[2 * (j - 1) + 1] : 0.0;
    const double al_prev = j > 0 ? coef[2 * (j - 1)] : 1.0;
    if (!(al > 0.0) || !(al_prev > 0.0) || !(be_prev >= 0.0)) return false;
    dg[j] = 1.0 / al + (j > 0 ? be_prev / al_prev : 0.0);
    if (j + 1 < kk) off[j] = std::sqrt(std::max(coef[2 * j + 1], 0.0)) / al;
  }
  tridiag_extremes(dg, off, lo, hi);
  return true;
}

// The inner solve's target at the Lemma 4.4 level: Lemma 4.2 bounds
// ||v|| <= sqrt(3 n mu) ||f||, and Lemma 4.4 needs ||v|| <= gamma sigma mu / 4,
// so ||f|| <= gamma sigma sqrt(mu) / (4 sqrt(3 n)).
inline double theory_inner_tol(double mu, long long n, double gamma, double sigma) {
  return gamma * sigma * std::sqrt(mu) / (4.0 * std::sqrt(3.0 * (double)n));
}

// The outer loop's stopping measures: the relative duality gap
// |c^T x - b^T y| / (1 + |c^T x|) and the relative residuals
// ||r_p|| / (1 + ||b||), ||r_d|| / (1 + ||c||); the solve stops when all three
// are at most tol.
struct StopMeasures {
  double gap, rp_rel, rd_rel;
};

inline StopMeasures stop_measures(double cx, double by, double rp2, double rd2, double bnorm, double cnorm) {
  return {std::fabs(cx - by) / (1.0 + std::fabs(cx)), std::sqrt(rp2) / (1.0 + bnorm),
          std::sqrt(rd2) / (1.0 + cnorm)};
}

inline bool stop_reached(const StopMeasures& s, double tol) {
  return s.gap <= tol && s.rp_rel <= tol && s.rd_rel <= tol;
}

}  // namespace lpk
