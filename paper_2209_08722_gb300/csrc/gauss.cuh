// The Gaussian sketch entries (Section 6), shared by the SIMT product, the
// tensor-core product and the correction-vector gather so that all three see
// bit-identical W'.
//
// Entry (j, k) of the draw for (k_iter, retry) has the flat index f = j*w + k
// and uses the draw at counter floor(f / 2) of the stream seeded with
// S = draw(draw(seed, 0), k_iter*16 + retry); its bits give
// u1 = (bits 41..63 + 1)/2^23 and u2 = (bits 18..40)/2^23 (both exact in
// FP32), and the entry is sqrt(-2 ln u1) cos(2 pi u2) / sqrt(w) for even f and
// sqrt(-2 ln u1) sin(2 pi u2) / sqrt(w) for odd f: both normals of one
// Box-Muller draw (FP32, CUDA's logf, sqrtf and sincospif).
// D is folded into the rows: W'_jk = fl32(fl32(d_j) * g_jk).
#pragma once
#include "internal.h"

namespace lpk {

__host__ __device__ inline uint64_t gauss_stream(uint64_t seed, long long k, int retry) {
  const uint64_t s_g = sm64_draw(seed, 0ull);
  return sm64_draw(s_g, (uint64_t)(k * kMaxRetry + retry));
}

// both normals of the draw at counter p: g0 (cosine, even flat index) and g1
// (sine, odd flat index), scaled by 1/sqrt(w)
__device__ __forceinline__ void gauss_pair(uint64_t s_kr, uint64_t p, float inv_sqrt_w, float* g0, float* g1) {
  const uint64_t v = sm64_draw(s_kr, p);
  // both integers are below 2^24, so the 32-bit conversions are exact
  const float u1 = (float)(uint32_t)((v >> 41) + 1ull) * 0x1p-23f;
  const float u2 = (float)(uint32_t)((v >> 18) & 0x7FFFFFull) * 0x1p-23f;
  const float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  *g0 = __fmul_rn(__fmul_rn(r, cs), inv_sqrt_w);
  *g1 = __fmul_rn(__fmul_rn(r, sn), inv_sqrt_w);
}

// the entry with flat index idx = j*w + k
__device__ __forceinline__ float gauss_entry(uint64_t s_kr, uint64_t idx, float inv_sqrt_w) {
  float g0, g1;
  gauss_pair(s_kr, idx >> 1, inv_sqrt_w, &g0, &g1);
  return (idx & 1ull) ? g1 : g0;
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
