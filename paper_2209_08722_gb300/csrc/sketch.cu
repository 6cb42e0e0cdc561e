// CountSketch A D W (Section 2, eq. pdprec; Algorithm 1 step 1) and the
// gather of the correction vector v (eq. compv).
//
// W (n x w) has s nonzeros per row: block b of width wb = w/s holds entry
// sign_b(i)/sqrt(s) at column b*wb + h_b(i), with (h_b(i), sign_b(i)) from the
// SplitMix64 counter-based generator (common.cuh).  W is never stored.
//
// The sketch is computed deterministically without global atomics: each CTA
// owns KB consecutive bucket columns of one block, scans the hashes of all n
// rows, compacts the rows that land in its buckets (in increasing i), and
// accumulates sign * d_i / sqrt(s) * a_i into FP64 shared-memory buckets.
// Bucket kl is owned by warp kl % 8, so every bucket is summed by one warp in
// increasing i: the result does not depend on scheduling.
#include "internal.h"

namespace lpk {

constexpr int kChunk = 2048;  // columns scanned per compaction round

template <typename TA>
__global__ void __launch_bounds__(kThreads) k_countsketch(
    const TA* __restrict__ A, int lda, int m, long long n, const double* __restrict__ dvec,
    int is_d2, uint64_t seed, long long k, int retry, int s_blocks, int wb, int KB,
    int groups_per_block, double* __restrict__ adw, int w) {
  constexpr int VEC = VecOf<TA>::N;
  extern __shared__ __align__(16) char smem[];
  double* acc = reinterpret_cast<double*>(smem);                  // [KB][lda]
  int* list_i = reinterpret_cast<int*>(acc + (size_t)KB * lda);  // [kChunk]
  float* list_v = reinterpret_cast<float*>(list_i + kChunk);     // scale (sign * d / sqrt s)
  short* list_k = reinterpret_cast<short*>(list_v + kChunk);     // local bucket
  __shared__ int warp_cnt[kWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x / groups_per_block;
  const int k0 = (blockIdx.x % groups_per_block) * KB;  // first bucket within block b
  const int kb = min(KB, wb - k0);
  if (kb <= 0) return;
  const int RV = lda / VEC;
  const double inv_sqrt_s = 1.0 / sqrt((double)s_blocks);

  for (int e = tid; e < KB * lda; e += blockDim.x) acc[e] = 0.0;
  __syncthreads();

  for (long long base = 0; base < n; base += kChunk) {
    int total = 0;
    // ---- compaction of the rows hitting [k0, k0 + kb) ----
    for (int sub = 0; sub < kChunk; sub += kThreads) {
      const long long i = base + sub + tid;
      bool hit = false;
      int kl = 0;
      float sg = 1.0f;
      if (i < n) {
        int col;
        cs_entry(seed, k, retry, b, i, wb, &col, &sg);
        kl = col - b * wb - k0;
        hit = (kl >= 0 && kl < kb);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) warp_cnt[warp] = __popc(bal);
      __syncthreads();
      int off = total;
      int tot = 0;
      for (int ww = 0; ww < kWarps; ++ww) {
        if (ww < warp) off += warp_cnt[ww];
        tot += warp_cnt[ww];
      }
      if (hit) {
        const int pos = off + __popc(bal & ((1u << lane) - 1u));
        list_i[pos] = (int)(i - base);
        list_v[pos] = sg;  // the FP64 scale d_i / sqrt(s) is applied when accumulating
        list_k[pos] = (short)kl;
      }
      total += tot;
      __syncthreads();
    }
    // ---- accumulation: warp (kl % kWarps) owns bucket kl ----
    for (int e = 0; e < total; ++e) {
      const int kl = list_k[e];
      if ((kl % kWarps) != warp) continue;
      const long long i = base + list_i[e];
      const double dv = is_d2 ? sqrt(dvec[i]) : dvec[i];
      const double scale = (double)list_v[e] * dv * inv_sqrt_s;
      const TA* col = A + (size_t)i * lda;
      double* dst = acc + (size_t)kl * lda;
      for (int rv = lane; rv < RV; rv += 32) {
        double av[VEC];
        ld16<double>(col + rv * VEC, av);
#pragma unroll
        for (int q = 0; q < VEC; ++q) dst[rv * VEC + q] = fma(av[q], scale, dst[rv * VEC + q]);
      }
    }
    __syncthreads();
  }
  // ---- write A D W (row-major m x w, FP64) ----
  for (int e = tid; e < kb * m; e += blockDim.x) {
    const int kl = e / m, i = e % m;
    adw[(size_t)i * w + b * wb + k0 + kl] = acc[(size_t)kl * lda + i];
  }
}

// v_i = sqrt(x_i s_i) / sqrt(s) * sum_b sign_b(i) u[col_b(i)]   (eq. compv with u = (ADW)^+ r)
__global__ void k_v_gather(long long n, const double* __restrict__ x, const double* __restrict__ s,
                           const double* __restrict__ u, uint64_t seed, long long k, int retry,
                           int s_blocks, int wb, double scale, double* __restrict__ v) {
  const double inv_sqrt_s = scale / sqrt((double)s_blocks);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < s_blocks; ++b) {
      int col;
      float sg;
      cs_entry(seed, k, retry, b, i, wb, &col, &sg);
      acc += (double)sg * u[col];
    }
    const double xs = s ? x[i] * s[i] : x[i];  // s == nullptr: x holds x o s
    v[i] = sqrt(xs) * inv_sqrt_s * acc;
  }
}

cudaError_t launch_countsketch(int dtype, const void* A, int lda, int m, long long n,
                               const double* dvec, int is_d2, uint64_t seed, long long k,
                               int retry, int s_blocks, int w, double* adw, int num_sms,
                               cudaStream_t st) {
  const int wb = w / s_blocks;
  const int esz = dtype == 0 ? 8 : (dtype == 1 ? 4 : 2);
  (void)esz;
  const int list_bytes = kChunk * (4 + 4 + 2);
  const int budget = 200 * 1024 - list_bytes;
  int kb_max = std::max(1, budget / (lda * 8));
  // aim for at least one CTA per SM
  int kb = (w + num_sms - 1) / num_sms;
  kb = std::max(1, std::min(kb, std::min(kb_max, wb)));
  const int groups_per_block = (wb + kb - 1) / kb;
  const int grid = groups_per_block * s_blocks;
  const int smem = kb * lda * 8 + list_bytes;
  cudaError_t e;
  if (dtype == 0) {
    e = cudaFuncSetAttribute(k_countsketch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_countsketch<double><<<grid, kThreads, smem, st>>>(
        static_cast<const double*>(A), lda, m, n, dvec, is_d2, seed, k, retry, s_blocks, wb, kb,
        groups_per_block, adw, w);
  } else if (dtype == 1) {
    e = cudaFuncSetAttribute(k_countsketch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_countsketch<float><<<grid, kThreads, smem, st>>>(
        static_cast<const float*>(A), lda, m, n, dvec, is_d2, seed, k, retry, s_blocks, wb, kb,
        groups_per_block, adw, w);
  } else {
    e = cudaFuncSetAttribute(k_countsketch<bf16raw>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_countsketch<bf16raw><<<grid, kThreads, smem, st>>>(
        static_cast<const bf16raw*>(A), lda, m, n, dvec, is_d2, seed, k, retry, s_blocks, wb, kb,
        groups_per_block, adw, w);
  }
  return cudaGetLastError();
}

cudaError_t launch_v_gather(long long n, const double* x, const double* s, const double* u,
                            uint64_t seed, long long k, int retry, int s_blocks, int w, double scale,
                            double* v, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_v_gather<<<grid, 256, 0, st>>>(n, x, s, u, seed, k, retry, s_blocks, w / s_blocks, scale, v);
  return cudaGetLastError();
}

}  // namespace lpk
