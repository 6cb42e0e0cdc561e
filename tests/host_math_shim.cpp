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
