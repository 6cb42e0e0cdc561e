// u = A diag(d2) A^T v accurate to FP64 level, computed with pairs of FP32
// numbers ("double-float": value = hi + lo, |lo| <= ulp(hi)/2).
//
// GB300's FP64 pipe runs at a small fraction of its FP32 pipe, so the FP64
// products of the outer iteration (the true-residual refresh of the normal
// equations, r = p - A D^2 A^T dy) are done on the FP32 pipe instead:
//   * a_ij is exact in FP32 (FP32 or BF16 storage);
//   * v_i (FP64) is split v = vh + vl; a*vh is formed exactly as p + e with an
//     FMA (error-free product), a*vl in FP32 (a term 2^-24 smaller);
//   * sums use the error-free TwoSum (Knuth), keeping the compensation in lo;
//   * t_j = d2_j (a_j^T v) in FP64 (one multiply per column), split again into
//     th + tl for the rank-1 update acc += a_j t_j, accumulated the same way.
// Relative error of each sum is about 2^-48, i.e. FP64-class for this use.
// Pipeline and reduction are those of k_adat_fused (warp-specialised bulk-copy
// ring; deterministic two-level FP64 reduction of the per-CTA partials).
#include "internal.h"
#include "stream_dev.cuh"
#include "df.cuh"

namespace lpk {

template <typename TA, int VPL, int CW>
__global__ void __launch_bounds__((CW + 1) * 32, 1) k_adat_df(const StreamArgs a) {
  constexpr int VEC = VecOf<TA>::N;
  extern __shared__ __align__(128) char smem[];
  const SmemLayout L = make_layout(a.lda, (int)sizeof(TA), a.nb, a.stages, 8);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* empty = full + a.stages;
  float* vh_s = reinterpret_cast<float*>(smem + L.v_off);
  float* vl_s = vh_s + a.lda;
  double* red = reinterpret_cast<double*>(smem + L.red_off);
  __shared__ int s_flag;
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RV = a.lda / VEC;
  const int S = a.stages;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], CW);
    }
    fence_mbar_init();
  }
  for (int i = tid; i < a.lda; i += blockDim.x) {
    const double v = (i < a.m) ? a.vin[i] : 0.0;
    const float h = (float)v;
    vh_s[i] = h;
    vl_s[i] = (float)(v - (double)h);
  }
  __syncthreads();

  float ah[VPL][VEC], al[VPL][VEC];
#pragma unroll
  for (int c = 0; c < VPL; ++c)
#pragma unroll
    for (int e = 0; e < VEC; ++e) ah[c][e] = al[c][e] = 0.0f;
  bool aborted = false;

  if (warp == CW) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < my_tiles; ++i) {
        const int st = i % S;
        if (i >= S && !mbar_wait(&empty[st], (uint32_t)(((i / S) - 1) & 1), a.err)) {
          aborted = true;
          break;
        }
        fence_proxy_async_smem();
        issue_tile<TA>(a, L, smem, full, st, (int)blockIdx.x + i * (int)gridDim.x);
        issued = i + 1;
      }
      if (aborted || *a.err != ERR_NONE)
        for (int j = (issued > S ? issued - S : 0); j < issued; ++j)
          mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), a.err);
    }
  } else {
    for (int i = 0; i < my_tiles; ++i) {
      const int st = i % S;
      if (!mbar_wait(&full[st], (uint32_t)((i / S) & 1), a.err)) {
        aborted = true;
        break;
      }
      const long long j0 = (long long)((int)blockIdx.x + i * (int)gridDim.x) * a.nb;
      const int ncols = (int)min((long long)a.nb, a.n - j0);
      const char* stage = smem + (size_t)st * L.stage_bytes;
      const TA* At = reinterpret_cast<const TA*>(stage);
      const double* d2t = reinterpret_cast<const double*>(stage + L.cv_off[0]);
      for (int jj = warp; jj < ncols; jj += CW) {
        const TA* col = At + (size_t)jj * a.lda;
        float av[VPL][VEC];
        float sh[2] = {0.0f, 0.0f}, sl[2] = {0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < VPL; ++c) {
          const int rv = c * 32 + lane;
          if (rv < RV) {
            ld16<float>(col + rv * VEC, av[c]);
#pragma unroll
            for (int e = 0; e < VEC; ++e)
              df_fma(av[c][e], vh_s[rv * VEC + e], vl_s[rv * VEC + e], sh[e & 1], sl[e & 1]);
          } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) av[c][e] = 0.0f;
          }
        }
        df_add(sh[0], sl[0], sh[1], sl[1]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, sh[0], o);
          const float ol = __shfl_xor_sync(0xffffffffu, sl[0], o);
          df_add(sh[0], sl[0], oh, ol);
        }
        const double t = d2t[jj] * ((double)sh[0] + (double)sl[0]);
        const float th = (float)t;
        const float tl = (float)(t - (double)th);
#pragma unroll
        for (int c = 0; c < VPL; ++c)
#pragma unroll
          for (int e = 0; e < VEC; ++e) df_fma(av[c][e], th, tl, ah[c][e], al[c][e]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  aborted = __syncthreads_or(aborted) != 0;
  // per-CTA partial in FP64: sum over the consumer warps through shared memory
  double* buf = reinterpret_cast<double*>(smem);
  if (warp < CW) {
#pragma unroll
    for (int c = 0; c < VPL; ++c) {
      const int rv = c * 32 + lane;
      if (rv < RV)
#pragma unroll
        for (int e = 0; e < VEC; ++e)
          buf[(size_t)warp * a.lda + rv * VEC + e] = (double)ah[c][e] + (double)al[c][e];
    }
  }
  __syncthreads();
  double* part = static_cast<double*>(a.partials) + (size_t)blockIdx.x * 2 * a.lda;
  for (int r = tid; r < a.lda; r += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < CW; ++w) s += buf[(size_t)w * a.lda + r];
    part[r] = aborted ? 0.0 : s;
  }
  if (a.epilogue == E_NONE) return;
  if (tree_reduce<double>(a, 1, &s_flag)) stream_epilogue<double>(a, 1, red);
}

namespace {
template <typename TA, int VPL, int CW>
cudaError_t df_launch(const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  auto k = k_adat_df<TA, VPL, CW>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k<<<grid, (CW + 1) * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename TA>
cudaError_t df_dispatch(int vpl, const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  switch (vpl) {
    case 1: return df_launch<TA, 1, 16>(a, grid, smem, st);
    case 2: return df_launch<TA, 2, 16>(a, grid, smem, st);
    case 4: return df_launch<TA, 4, 16>(a, grid, smem, st);
    case 8: return df_launch<TA, 8, 8>(a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

// Largest m served: VPL <= 8 (FP32: 1024 rows, BF16: 2048 rows); the caller
// uses the FP64 streaming kernel beyond that.
bool adat_df_supported(int lda, int esz) {
  const int vpl = fused_vpl(lda, esz);
  return vpl >= 1 && vpl <= 8;
}

cudaError_t launch_adat_df(int dtype, const StreamArgs& a, const StreamPlan& p, cudaStream_t st) {
  const int esz = dtype == 1 ? 4 : 2;
  const int vpl = fused_vpl(a.lda, esz);
  if (dtype == 1) return df_dispatch<float>(vpl, a, p.grid, p.smem8, st);
  if (dtype == 2) return df_dispatch<bf16raw>(vpl, a, p.grid, p.smem8, st);
  return cudaErrorInvalidValue;
}

}  // namespace lpk
