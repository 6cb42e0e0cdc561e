// Gaussian sketch (Section 6): A D W_G with W_G (n x w) iid N(0, 1/w), drawn
// on the fly from the SplitMix64 counter-based generator -- W_G is never
// stored.  Entry (j, k) of the draw for (k_iter, retry) has the flat index
// f = j*w + k and uses the draw at counter floor(f/2) of the stream seeded
// with S = draw(draw(seed, 0), k_iter*16 + retry); its bits give
// u1 = (bits 41..63 + 1)/2^23, u2 = (bits 18..40)/2^23 (exact in FP32) and
// g = sqrt(-2 ln u1) cos(2 pi u2) / sqrt(w) for even f, the sine for odd f
// (both Box-Muller outputs, FP32).
//
// D is folded into the rows of W: W'_jk = fl32(fl32(d_j) * g_jk), so that
// A D W = A W' and the correction vector of eq. (compv) is
// v_j = sqrt(x_j s_j) / d_j * (W' u)_j with the same W'.
//
// k_gauss_sketch: FP32 SIMT tiled product with split-K: each CTA owns a
// 128 x 64 output tile and a slice of the n columns of A, regenerates its W'
// tile in shared memory and adds its FP32 tile into the FP64 result with
// atomics.  It serves FP64 storage and is the cross-check of the tensor-core
// version in gauss_tc.cu, which computes the same product.
#include "gauss.cuh"

namespace lpk {

constexpr int GBM = 128, GBN = 64, GBK = 16;

template <typename TA>
__global__ void __launch_bounds__(256) k_gauss_sketch(const TA* __restrict__ A, int lda, int m,
                                                      long long n, const double* __restrict__ dvec,
                                                      int is_d2, uint64_t s_kr, int w, float inv_sqrt_w,
                                                      long long kper, double* __restrict__ adw) {
  __shared__ float As[GBK][GBM];
  __shared__ float Ws[GBK][GBN];
  __shared__ float ds[GBK];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.x * GBM, k0 = blockIdx.y * GBN;
  const long long j0 = blockIdx.z * kper;
  const long long j1 = min(n, j0 + kper);
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  for (long long jb = j0; jb < j1; jb += GBK) {
    // A tile: GBK columns x GBM rows (each column contiguous in memory)
    for (int e = tid; e < GBK * GBM; e += 256) {
      const int jj = e / GBM, ii = e % GBM;
      const long long j = jb + jj;
      float av = 0.0f;
      if (j < j1 && i0 + ii < m) {
        if (sizeof(TA) == 8) av = (float)reinterpret_cast<const double*>(A)[(size_t)j * lda + i0 + ii];
        else if (sizeof(TA) == 4) av = reinterpret_cast<const float*>(A)[(size_t)j * lda + i0 + ii];
        else av = __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(A)[(size_t)j * lda + i0 + ii] << 16);
      }
      As[jj][ii] = av;
    }
    if (tid < GBK) ds[tid] = jb + tid < j1 ? gauss_dval(dvec, jb + tid, is_d2) : 0.0f;
    __syncthreads();
    // W' tile: GBK rows x GBN sketch columns
    for (int e = tid; e < GBK * GBN; e += 256) {
      const int jj = e / GBN, kk = e % GBN;
      const long long j = jb + jj;
      float wv = 0.0f;
      if (j < j1 && k0 + kk < w)
        wv = gauss_wprime(ds[jj], s_kr, (uint64_t)j * w + k0 + kk, inv_sqrt_w);
      Ws[jj][kk] = wv;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < GBK; ++jj) {
      float a[8], b[4];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = As[jj][ty * 8 + q];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Ws[jj][tx * 4 + q];
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int i = i0 + ty * 8 + p;
    if (i >= m) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + tx * 4 + q;
      if (k < w) atomicAdd(&adw[(size_t)i * w + k], (double)acc[p][q]);
    }
  }
}

// v_j = scale * sqrt(xs_j) / d_j * sum_k W'_jk u_k   (one warp per j; the sum in FP64)
__global__ void __launch_bounds__(256) k_gauss_v(long long n, const double* __restrict__ x,
                                                 const double* __restrict__ s,
                                                 const double* __restrict__ dvec, int is_d2,
                                                 const double* __restrict__ u, uint64_t s_kr, int w,
                                                 float inv_sqrt_w, double scale, double* __restrict__ v) {
  extern __shared__ double u_s[];
  for (int k = threadIdx.x; k < w; k += blockDim.x) u_s[k] = u[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long j = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
    const float dj = gauss_dval(dvec, j, is_d2);
    double acc = 0.0;
    for (int k = lane; k < w; k += 32)
      acc = fma((double)__fmul_rn(dj, gauss_entry(s_kr, (uint64_t)j * w + k, inv_sqrt_w)), u_s[k], acc);
    acc = warp_sum(acc);
    if (lane == 0) {
      const double xs = s ? x[j] * s[j] : x[j];
      v[j] = scale * sqrt(xs) / (double)dj * acc;
    }
  }
}

cudaError_t launch_gauss_sketch(int dtype, const void* A, int lda, int m, long long n,
                                const double* dvec, int is_d2, uint64_t seed, long long k, int retry,
                                int w, double* adw, int tensor, int* err, int num_sms,
                                cudaStream_t st) {
  const uint64_t s_kr = gauss_stream(seed, k, retry);
  const float inv_sqrt_w = (float)(1.0 / sqrt((double)w));
  if (tensor && (dtype == 1 || dtype == 2))
    return launch_gauss_tc(dtype, A, lda, m, n, dvec, is_d2, s_kr, w, inv_sqrt_w, adw, err, num_sms, st);
  cudaError_t e = cudaMemsetAsync(adw, 0, sizeof(double) * (size_t)m * w, st);
  if (e != cudaSuccess) return e;
  const int gx = (m + GBM - 1) / GBM, gy = (w + GBN - 1) / GBN;
  long long ks = std::max<long long>(1, std::min<long long>((n + 4095) / 4096, 64));
  const long long kper = ((n + ks - 1) / ks + GBK - 1) / GBK * GBK;
  ks = (n + kper - 1) / kper;
  dim3 grid(gx, gy, (unsigned)ks);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (dtype == 0)
    k_gauss_sketch<double><<<grid, 256, 0, st>>>(static_cast<const double*>(A), lda, m, n, dvec, is_d2,
                                                  s_kr, w, inv_sqrt_w, kper, adw);
  else if (dtype == 1)
    k_gauss_sketch<float><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, m, n, dvec, is_d2,
                                                 s_kr, w, inv_sqrt_w, kper, adw);
  else
    k_gauss_sketch<bf16raw><<<grid, 256, 0, st>>>(static_cast<const bf16raw*>(A), lda, m, n, dvec,
                                                   is_d2, s_kr, w, inv_sqrt_w, kper, adw);
  return cudaGetLastError();
}

cudaError_t launch_gauss_v(long long n, const double* x, const double* s, const double* dvec,
                           int is_d2, const double* u, uint64_t seed, long long k, int retry, int w,
                           double scale, double* v, int num_sms, cudaStream_t st) {
  const uint64_t s_kr = gauss_stream(seed, k, retry);
  const float inv_sqrt_w = (float)(1.0 / sqrt((double)w));
  const int smem = w * 8;
  cudaError_t e = ensure_smem((const void*)k_gauss_v, smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 7) / 8, num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_gauss_v<<<grid, 256, smem, st>>>(n, x, s, dvec, is_d2, u, s_kr, w, inv_sqrt_w, scale, v);
  return cudaGetLastError();
}

}  // namespace lpk
