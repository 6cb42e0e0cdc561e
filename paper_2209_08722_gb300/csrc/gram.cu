// Gram matrix Q = (ADW)(ADW)^T of the sketch (Algorithm 1 step 2: the factor
// of Q gives the preconditioner) in double-float arithmetic on the FP32 pipe.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the m x m x w
// contraction is carried out on pairs of FP32 numbers instead:
//   1. k_split_df: X = ADW (FP64, row-major m x w) -> X_hi + X_lo, two FP32
//      arrays with X_hi = fl32(X), X_lo = fl32(X - X_hi) (|X - X_hi - X_lo| <=
//      2^-48 |X|);
//   2. k_gram_df: upper-triangle 64 x 64 tiles of X X^T with split-K; every
//      product (a_hi + a_lo)(b_hi + b_lo) is formed with an exact FP32 product
//      and its error term, and summed in double-float (relative error ~2^-46
//      of sum |x_ik x_jk|, the order of an FP64 GEMM's bound);
//   3. k_gram_reduce: the split-K partials summed in slice order (the result is
//      bitwise reproducible) into the upper triangle of the column-major m x m
//      output, in FP64.
#include "internal.h"
#include "df.cuh"

#include <atomic>

namespace lpk {

namespace {
constexpr int GT = 64;        // output tile
constexpr int GK = 32;        // k per shared-memory chunk
constexpr int GTHREADS = 256; // 16 x 16 threads, 4 x 4 outputs each
}  // namespace

__global__ void __launch_bounds__(256) k_split_df(const double* __restrict__ x, long long count,
                                                  float* __restrict__ xh, float* __restrict__ xl) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float hi = (float)v;
    xh[e] = hi;
    xl[e] = (float)(v - (double)hi);
  }
}

// tile t of the upper triangle (row block bi <= column block bj), slice z of k
__global__ void __launch_bounds__(GTHREADS) k_gram_df(const float* __restrict__ xh,
                                                      const float* __restrict__ xl, int m, int w,
                                                      int nt, int kper, float2* __restrict__ part) {
  // [k][row], rows padded to 68 floats (16-byte aligned rows, fewer bank conflicts)
  __shared__ __align__(16) float ah[GK][GT + 4], al[GK][GT + 4], bh[GK][GT + 4], bl[GK][GT + 4];
  // tile index -> (bi, bj), bi <= bj, row-major over the upper triangle
  int t = blockIdx.x, bi = 0;
  while (t >= nt - bi) {
    t -= nt - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int i0 = bi * GT, j0 = bj * GT;
  const int k0 = blockIdx.y * kper, k1 = min(w, k0 + kper);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      sh[a][b] = 0.0f;
      sl[a][b] = 0.0f;
    }
  for (int kb = k0; kb < k1; kb += GK) {
    // stage 64 rows x 32 k of both operands, transposed to [k][row]; each
    // thread reads 4 consecutive k of one row (8 threads per 128-byte row piece)
    for (int e = tid; e < GT * (GK / 4); e += GTHREADS) {
      const int r = e / (GK / 4), k4 = (e % (GK / 4)) * 4;
      const int ia = i0 + r, ib = j0 + r;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = kb + k4 + q;
        const bool ka = k < k1;
        ah[k4 + q][r] = (ka && ia < m) ? xh[(size_t)ia * w + k] : 0.0f;
        al[k4 + q][r] = (ka && ia < m) ? xl[(size_t)ia * w + k] : 0.0f;
        bh[k4 + q][r] = (ka && ib < m) ? xh[(size_t)ib * w + k] : 0.0f;
        bl[k4 + q][r] = (ka && ib < m) ? xl[(size_t)ib * w + k] : 0.0f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a_h = *reinterpret_cast<const float4*>(&ah[kk][ty * 4]);
      const float4 a_l = *reinterpret_cast<const float4*>(&al[kk][ty * 4]);
      const float4 b_h = *reinterpret_cast<const float4*>(&bh[kk][tx * 4]);
      const float4 b_l = *reinterpret_cast<const float4*>(&bl[kk][tx * 4]);
      const float avh[4] = {a_h.x, a_h.y, a_h.z, a_h.w}, avl[4] = {a_l.x, a_l.y, a_l.z, a_l.w};
      const float bvh[4] = {b_h.x, b_h.y, b_h.z, b_h.w}, bvl[4] = {b_l.x, b_l.y, b_l.z, b_l.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // (ah + al)(bh + bl) = p + e up to the dropped al*bl (2^-48 relative)
          const float p = __fmul_rn(avh[a], bvh[b]);
          float e = fmaf(avh[a], bvh[b], -p);
          e = fmaf(avh[a], bvl[b], e);
          e = fmaf(avl[a], bvh[b], e);
          float s, q;
          two_sum(sh[a][b], p, s, q);
          sh[a][b] = s;
          sl[a][b] = __fadd_rn(sl[a][b], __fadd_rn(q, e));
        }
      if ((kk & 7) == 7) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) df_renorm(sh[a][b], sl[a][b]);
      }
    }
    __syncthreads();
  }
  float2* out = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (GT * GT);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) out[(ty * 4 + a) * GT + tx * 4 + b] = make_float2(sh[a][b], sl[a][b]);
}

// G (column-major m x m, upper triangle) = sum over slices, in slice order
__global__ void __launch_bounds__(256) k_gram_reduce(const float2* __restrict__ part, int m, int nt,
                                                     int ntiles, int ks, double* __restrict__ g) {
  const long long total = (long long)ntiles * GT * GT;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int tile = (int)(e / (GT * GT)), loc = (int)(e % (GT * GT));
    int t = tile, bi = 0;
    while (t >= nt - bi) {
      t -= nt - bi;
      ++bi;
    }
    const int bj = bi + t;
    const int i = bi * GT + loc / GT, j = bj * GT + loc % GT;
    if (i >= m || j >= m || i > j) continue;
    float2 v = part[e];
    float hi = v.x, lo = v.y;
    for (int z = 1; z < ks; ++z) {
      const float2 o = part[(size_t)z * total + e];
      df_add(hi, lo, o.x, o.y);
    }
    g[(size_t)j * m + i] = (double)hi + (double)lo;
  }
}

size_t gram_df_scratch_floats(int m, int w, int num_sms) {
  const int nt = (m + GT - 1) / GT;
  const int ntiles = nt * (nt + 1) / 2;
  int ks, kper;
  gram_df_split(m, w, num_sms, &ks, &kper);
  return (size_t)2 * m * w + (size_t)2 * ks * ntiles * GT * GT;
}

// CTAs of k_gram_df resident per SM (occupancy query once per process; 3 if
// the query fails)
static int gram_ctas_per_sm() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_relaxed);
  if (v == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gram_df, GTHREADS, 0) != cudaSuccess || b <= 0) {
      cudaGetLastError();
      b = 3;
    }
    v = b;
    cached.store(v, std::memory_order_relaxed);
  }
  return v;
}

// Split of K = w into ks slices of kper (a multiple of GK, at least 128): the
// run time goes as (waves of ntiles * ks CTAs over the resident slots) / ks,
// so ks is the smallest that minimises it (a last, partly filled wave costs a
// whole wave of CTAs that each do 1/ks of the work)
void gram_df_split(int m, int w, int num_sms, int* ks_out, int* kper_out) {
  const int nt = (m + GT - 1) / GT;
  const long long ntiles = (long long)nt * (nt + 1) / 2;
  const long long slots = (long long)std::max(1, num_sms) * gram_ctas_per_sm();
  const int ks_max = std::max(1, std::min(64, w / 128));
  int best = 1;
  double best_t = 0.0;
  for (int ks = 1; ks <= ks_max; ++ks) {
    const double t = (double)((ntiles * ks + slots - 1) / slots) / ks + 0.01 * ks;  // + reduction traffic
    if (ks == 1 || t < best_t - 1e-12) {
      best = ks;
      best_t = t;
    }
  }
  const int kper = ((w + best - 1) / best + GK - 1) / GK * GK;
  *ks_out = (w + kper - 1) / kper;
  *kper_out = kper;
}

cudaError_t launch_gram_df(const double* x, int m, int w, float* scratch, double* g, int num_sms,
                           cudaStream_t st) {
  const int nt = (m + GT - 1) / GT;
  const int ntiles = nt * (nt + 1) / 2;
  int ks, kper;
  gram_df_split(m, w, num_sms, &ks, &kper);
  float* xh = scratch;
  float* xl = scratch + (size_t)m * w;
  float2* part = reinterpret_cast<float2*>(scratch + (size_t)2 * m * w);
  const long long count = (long long)m * w;
  const int g1 = (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, (long long)num_sms * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_split_df<<<g1, 256, 0, st>>>(x, count, xh, xl);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_gram_df<<<dim3((unsigned)ntiles, (unsigned)ks), GTHREADS, 0, st>>>(xh, xl, m, w, nt, kper, part);
  const long long total = (long long)ntiles * GT * GT;
  const int g3 = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, (long long)num_sms * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_gram_reduce<<<g3, 256, 0, st>>>(part, m, nt, ntiles, ks, g);
  return cudaGetLastError();
}

}  // namespace lpk
