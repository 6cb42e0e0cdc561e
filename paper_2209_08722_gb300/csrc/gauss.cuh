// The Gaussian sketch entries (Section 6), shared by the SIMT product, the
// tensor-core product and the correction-vector gather so that all three see
// bit-identical W'.
//
// Entry (j, k) of the draw for (k_iter, retry) uses counter j*w + k of the
// stream seeded with S = draw(draw(seed, 0), k_iter*16 + retry); its bits give
// u1 = (bits 41..63 + 1)/2^23 and u2 = (bits 18..40)/2^23 (both exact in
// FP32), and g = sqrt(-2 ln u1) cos(2 pi u2) / sqrt(w) (Box-Muller, FP32).
// D is folded into the rows: W'_jk = fl32(fl32(d_j) * g_jk).
#pragma once
#include "internal.h"

namespace lpk {

__host__ __device__ inline uint64_t gauss_stream(uint64_t seed, long long k, int retry) {
  const uint64_t s_g = sm64_draw(seed, 0ull);
  return sm64_draw(s_g, (uint64_t)(k * kMaxRetry + retry));
}

__device__ __forceinline__ float gauss_entry(uint64_t s_kr, uint64_t idx, float inv_sqrt_w) {
  const uint64_t v = sm64_draw(s_kr, idx);
  // both integers are below 2^24, so the 32-bit conversions are exact
  const float u1 = (float)(uint32_t)((v >> 41) + 1ull) * 0x1p-23f;
  const float u2 = (float)(uint32_t)((v >> 18) & 0x7FFFFFull) * 0x1p-23f;
  return __fmul_rn(__fmul_rn(sqrtf(-2.0f * logf(u1)), cospif(2.0f * u2)), inv_sqrt_w);
}

__device__ __forceinline__ float gauss_dval(const double* dvec, long long j, int is_d2) {
  const double d = dvec[j];
  return (float)(is_d2 ? sqrt(d) : d);
}

// dj = gauss_dval(dvec, j, is_d2), computed once per column j by the caller
__device__ __forceinline__ float gauss_wprime(float dj, uint64_t s_kr, uint64_t idx, float inv_sqrt_w) {
  return __fmul_rn(dj, gauss_entry(s_kr, idx, inv_sqrt_w));
}

}  // namespace lpk
