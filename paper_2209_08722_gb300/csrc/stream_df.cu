// Column-streaming passes over A with FP64-class accuracy computed in pairs
// of FP32 numbers ("double-float": value = hi + lo, |lo| <= ulp(hi)/2).
//
// GB300's FP64 pipe runs at a small fraction of its FP32 pipe, so the FP64
// passes of an outer iteration run on the FP32 pipe instead:
//   M_ADAT  u = A diag(d2) A^T v           (the true-residual refresh of the
//                                           normal equations, eq. normal)
//   M_RESID r_d = A^T y + s - c, d2 = x/s, r_p = A x - b and the right-hand
//           side p = A(x - sigma mu/s - d2 r_d) - r_p    (Alg. 3 steps 3-4)
//   M_DIR   ds = -r_d - A^T dy, dx = -x + sigma mu/s - d2 ds - v/s
//                                          (eqs. delshat, delxhat)
// Arithmetic:
//   * a_ij is exact in FP32 (FP32 or BF16 storage);
//   * the m-vector v (FP64) is split once into vh + vl in shared memory;
//     a * vh is formed exactly as p + e with an FMA, a * vl in FP32;
//   * sums use the error-free TwoSum, keeping the compensation in lo;
//   * per column, lane 0 forms the column scalars (d2_j (a_j^T v), or the
//     residual/direction formulas) in FP64, splits them into FP32 pairs and
//     broadcasts them; the rank-1 updates acc += a_j t_j use the same exact
//     products.
// The relative error of each sum is about 2^-46 of the sum of |terms|.
// Pipeline: one producer warp issues bulk copies of column tiles into a ring
// of stages; CW consumer warps take whole columns (warp-per-column), keep the
// per-row accumulators of their columns in registers, and combine them at the
// end in double-float through shared memory; the per-CTA partials then go
// through the deterministic two-level FP64 reduction and the mode epilogue
// shared with the FP64 streaming kernel.
#include "internal.h"
#include "stream_dev.cuh"
#include "df.cuh"

namespace lpk {

namespace {
__device__ __forceinline__ void split_df(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}
}  // namespace

template <typename TA, int VPL, int CW, int MODE>
__global__ void __launch_bounds__((CW + 1) * 32, 1) k_stream_df(const StreamArgs a) {
  constexpr int VEC = VecOf<TA>::N;
  constexpr int NACC = (MODE == M_RESID) ? 2 : ((MODE == M_ADAT) ? 1 : 0);
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
  const double sigma_mu = (MODE == M_RESID || MODE == M_DIR) ? a.sigma * a.sc->mu : 0.0;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], CW);
    }
    fence_mbar_init();
  }
  for (int i = tid; i < a.lda; i += blockDim.x) split_df((i < a.m) ? a.vin[i] : 0.0, vh_s[i], vl_s[i]);
  __syncthreads();

  float ah[NACC > 0 ? VPL : 1][VEC], al[NACC > 0 ? VPL : 1][VEC];
  float bh[NACC > 1 ? VPL : 1][VEC], bl[NACC > 1 ? VPL : 1][VEC];
#pragma unroll
  for (int c = 0; c < (NACC > 0 ? VPL : 1); ++c)
#pragma unroll
    for (int e = 0; e < VEC; ++e) ah[c][e] = al[c][e] = 0.0f;
#pragma unroll
  for (int c = 0; c < (NACC > 1 ? VPL : 1); ++c)
#pragma unroll
    for (int e = 0; e < VEC; ++e) bh[c][e] = bl[c][e] = 0.0f;
  double cred0 = 0.0, cred1 = 0.0;  // column reductions (lane 0)
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
        // ---- per-column scalars, in FP64 on lane 0 ----
        float t0h = 0.0f, t0l = 0.0f, t1h = 0.0f, t1l = 0.0f;
        if (lane == 0) {
          const double dot = (double)sh[0] + (double)sl[0];
          const long long j = j0 + jj;
          double t0 = 0.0, t1 = 0.0;
          if (MODE == M_ADAT) {
            t0 = cv_at(stage, L, a, 0, jj) * dot;
          } else if (MODE == M_RESID) {
            const double x = cv_at(stage, L, a, 0, jj);
            const double s = cv_at(stage, L, a, 1, jj);
            const double c = cv_at(stage, L, a, 2, jj);
            const double rd = dot + s - c;
            const double d2 = x / s;
            a.out_col[0][j] = rd;
            a.out_col[1][j] = d2;
            a.out_colf[j] = (float)d2;
            t0 = x;
            t1 = a.feasible ? (x - sigma_mu / s) : (x - sigma_mu / s - d2 * rd);
            cred0 += rd * rd;
            cred1 += c * x;
          } else if (MODE == M_DIR) {
            const double x = cv_at(stage, L, a, 0, jj);
            const double s = cv_at(stage, L, a, 1, jj);
            const double v = cv_at(stage, L, a, 2, jj);
            const double rd = a.feasible ? 0.0 : cv_at(stage, L, a, 3, jj);
            const double ds = -rd - dot;
            const double dx = -x + sigma_mu / s - (x / s) * ds - v / s;
            a.out_col[0][j] = dx;
            a.out_col[1][j] = ds;
            cred0 += x * ds + s * dx;
            cred1 += dx * ds;
          }
          if (NACC > 0) split_df(t0, t0h, t0l);
          if (NACC > 1) split_df(t1, t1h, t1l);
        }
        if (NACC > 0) {
          t0h = __shfl_sync(0xffffffffu, t0h, 0);
          t0l = __shfl_sync(0xffffffffu, t0l, 0);
#pragma unroll
          for (int c = 0; c < VPL; ++c)
#pragma unroll
            for (int e = 0; e < VEC; ++e) df_fma(av[c][e], t0h, t0l, ah[c][e], al[c][e]);
        }
        if (NACC > 1) {
          t1h = __shfl_sync(0xffffffffu, t1h, 0);
          t1l = __shfl_sync(0xffffffffu, t1l, 0);
#pragma unroll
          for (int c = 0; c < VPL; ++c)
#pragma unroll
            for (int e = 0; e < VEC; ++e) df_fma(av[c][e], t1h, t1l, bh[c][e], bl[c][e]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  aborted = __syncthreads_or(aborted) != 0;
  // ---- per-CTA partials: sum over the consumer warps in double-float through
  // shared memory (the stage area is free), one FP64 conversion per row ----
  float2* buf = reinterpret_cast<float2*>(smem);
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    if (warp < CW) {
#pragma unroll
      for (int c = 0; c < VPL; ++c) {
        const int rv = c * 32 + lane;
        if (rv < RV)
#pragma unroll
          for (int e = 0; e < VEC; ++e)
            buf[(size_t)warp * a.lda + rv * VEC + e] =
                k == 0 ? make_float2(ah[c][e], al[c][e])
                       : make_float2(bh[NACC > 1 ? c : 0][e], bl[NACC > 1 ? c : 0][e]);
      }
    }
    __syncthreads();
    double* part = static_cast<double*>(a.partials) + (size_t)blockIdx.x * 2 * a.lda + (size_t)k * a.lda;
    for (int r = tid; r < a.lda; r += blockDim.x) {
      float h = buf[r].x, l = buf[r].y;
      for (int w = 1; w < CW; ++w) df_add(h, l, buf[(size_t)w * a.lda + r].x, buf[(size_t)w * a.lda + r].y);
      part[r] = aborted ? 0.0 : (double)h + (double)l;
    }
    __syncthreads();
  }
  if (a.red_partials) {
    const double r0 = block_sum(lane == 0 && warp < CW ? cred0 : 0.0, red);
    const double r1 = block_sum(lane == 0 && warp < CW ? cred1 : 0.0, red);
    if (tid == 0) {
      a.red_partials[2 * blockIdx.x] = r0;
      a.red_partials[2 * blockIdx.x + 1] = r1;
    }
  }
  if (a.epilogue == E_NONE) return;
  if (tree_reduce<double>(a, NACC, &s_flag)) stream_epilogue<double>(a, NACC, red);
}

namespace {
// register budget: 17 warps (16 consumers) leave 96 registers per thread (a
// scheduler holds 5 warps), 9 warps 168.  Each accumulator set costs two
// registers per accumulated element, the column slice one; so 16 consumers
// take up to 16 elements with one set (4 with two), 8 consumers up to 32 with
// one set (16 with two).
template <int MODE>
constexpr int df_nacc() {
  return MODE == M_RESID ? 2 : (MODE == M_ADAT ? 1 : 0);
}

template <int MODE>
constexpr int df_cw(int elems) {
  return df_nacc<MODE>() == 2 ? (elems <= 4 ? 16 : 8) : (elems <= 16 ? 16 : 8);
}

template <int MODE>
constexpr bool df_fits(int elems) {
  return df_nacc<MODE>() == 2 ? elems <= 16 : elems <= 32;
}

template <typename TA, int VPL, int MODE>
cudaError_t df_launch(const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  constexpr int VEC = VecOf<TA>::N;
  if constexpr (!df_fits<MODE>(VPL * VEC)) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int CW = df_cw<MODE>(VPL * VEC);
    auto k = k_stream_df<TA, VPL, CW, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k<<<grid, (CW + 1) * 32, smem, st>>>(a);
    return cudaGetLastError();
  }
}

template <typename TA, int MODE>
cudaError_t df_dispatch(int vpl, const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  switch (vpl) {
    case 1: return df_launch<TA, 1, MODE>(a, grid, smem, st);
    case 2: return df_launch<TA, 2, MODE>(a, grid, smem, st);
    case 4: return df_launch<TA, 4, MODE>(a, grid, smem, st);
    case 8: return df_launch<TA, 8, MODE>(a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t df_mode(int dtype, int vpl, const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  if (dtype == 1) return df_dispatch<float, MODE>(vpl, a, grid, smem, st);
  if (dtype == 2) return df_dispatch<bf16raw, MODE>(vpl, a, grid, smem, st);
  return cudaErrorInvalidValue;
}
}  // namespace

// FP32/BF16 storage with VPL <= 8; the accumulator sets must fit the register
// budget and the consumers' combine buffer (CW x lda pairs) the stage ring.
bool stream_df_supported(int mode, int lda, int esz, const StreamPlan& p) {
  if (esz != 4 && esz != 2) return false;
  const int vpl = fused_vpl(lda, esz);
  if (vpl < 1 || vpl > 8) return false;
  const int elems = vpl * (16 / esz);
  int cw;
  if (mode == M_ADAT) {
    if (!df_fits<M_ADAT>(elems)) return false;
    cw = df_cw<M_ADAT>(elems);
  } else if (mode == M_RESID) {
    if (!df_fits<M_RESID>(elems)) return false;
    cw = df_cw<M_RESID>(elems);
  } else if (mode == M_DIR) {
    if (!df_fits<M_DIR>(elems)) return false;
    cw = df_cw<M_DIR>(elems);
  } else {
    return false;
  }
  const SmemLayout L = make_layout(lda, esz, p.nb, p.stages, 8);
  return (long long)cw * lda * 8 <= (long long)p.stages * L.stage_bytes && p.smem8 <= 227 * 1024;
}

cudaError_t launch_stream_df(int dtype, int mode, const StreamArgs& a, const StreamPlan& p,
                             cudaStream_t st) {
  const int esz = dtype == 1 ? 4 : 2;
  const int vpl = fused_vpl(a.lda, esz);
  if (mode == M_ADAT) return df_mode<M_ADAT>(dtype, vpl, a, p.grid, p.smem8, st);
  if (mode == M_RESID) return df_mode<M_RESID>(dtype, vpl, a, p.grid, p.smem8, st);
  if (mode == M_DIR) return df_mode<M_DIR>(dtype, vpl, a, p.grid, p.smem8, st);
  return cudaErrorInvalidValue;
}

}  // namespace lpk
