// Test shim: exposes the solver's host-side numerical helpers
// (paper_2209_08722_gb300/csrc/host_math.h) with a C ABI so that the CPU
// tests can call them through ctypes.  Compiled by tests/test_host_math.py.
#include "host_math.h"

extern "C" int shim_lanczos_extremes(const double* coef, int kk, double* lo, double* hi) {
  return lpk::lanczos_extremes(coef, kk, lo, hi) ? 1 : 0;
}

extern "C" void shim_tridiag_extremes(const double* dg, const double* off, int k, double* lo, double* hi) {
  std::vector<double> d(dg, dg + k), o(off, off + (k > 0 ? k - 1 : 0));
  lpk::tridiag_extremes(d, o, lo, hi);
}

extern "C" double shim_theory_inner_tol(double mu, long long n, double gamma, double sigma) {
  return lpk::theory_inner_tol(mu, n, gamma, sigma);
}

extern "C" int shim_stop(double cx, double by, double rp2, double rd2, double bnorm, double cnorm, double tol,
                         double* out3) {
  const lpk::StopMeasures s = lpk::stop_measures(cx, by, rp2, rd2, bnorm, cnorm);
  out3[0] = s.gap;
  out3[1] = s.rp_rel;
  out3[2] = s.rd_rel;
  return lpk::stop_reached(s, tol) ? 1 : 0;
}
