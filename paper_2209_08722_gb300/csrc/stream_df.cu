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
//   * the per-column inputs (d2, or x, s, c / x, s, v, r_d) arrive as FP32
//     pairs (packed from the FP64 vectors by k_df_pack) and lane 0 forms the
//     column scalars (d2_j (a_j^T v), or the residual/direction formulas) in
//     double-float and broadcasts them; the rank-1 updates acc += a_j t_j use
//     the same exact products.  Per-column outputs are written as pairs and
//     unpacked to FP64 (with the column sums the epilogues need) afterwards.
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

// per-column input q of the current tile, stored as FP32 pairs
__device__ __forceinline__ dfl cv_df(const char* stage, const SmemLayout& L, int q, int jj) {
  const float2 v = reinterpret_cast<const float2*>(stage + L.cv_off[q])[jj];
  return {v.x, v.y};
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
  pdl_wait();
  pdl_trigger();
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RV = a.lda / VEC;
  const int S = a.stages;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  dfl smu = {0.0f, 0.0f};  // sigma mu as a pair (one FP64 product per CTA)
  if (MODE == M_RESID || MODE == M_DIR) {
    const double v = a.sigma * a.sc->mu;
    smu.h = (float)v;
    smu.l = (float)(v - (double)smu.h);
  }

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
    // this lane's slice of v as pairs, in registers for the whole stream
    float vrh[VPL][VEC], vrl[VPL][VEC];
#pragma unroll
    for (int c = 0; c < VPL; ++c)
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int rv = c * 32 + lane;
        vrh[c][e] = (rv < RV) ? vh_s[rv * VEC + e] : 0.0f;
        vrl[c][e] = (rv < RV) ? vl_s[rv * VEC + e] : 0.0f;
      }
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
        float sh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < VPL; ++c) {
          const int rv = c * 32 + lane;
          if (rv < RV) {
            ld16<float>(col + rv * VEC, av[c]);
#pragma unroll
            for (int e = 0; e < VEC; ++e) df_fma(av[c][e], vrh[c][e], vrl[c][e], sh[e & 3], sl[e & 3]);
          } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) av[c][e] = 0.0f;
          }
        }
        df_add(sh[0], sl[0], sh[1], sl[1]);
        df_add(sh[2], sl[2], sh[3], sl[3]);
        df_add(sh[0], sl[0], sh[2], sl[2]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, sh[0], o);
          const float ol = __shfl_xor_sync(0xffffffffu, sl[0], o);
          df_add(sh[0], sl[0], oh, ol);
        }
        // ---- per-column scalars, in double-float on lane 0 (the FP64 pipe
        // would serialise them: a one-lane FP64 instruction costs the pipe as
        // much as a full warp's) ----
        float t0h = 0.0f, t0l = 0.0f, t1h = 0.0f, t1l = 0.0f;
        if (lane == 0) {
          const dfl dot = dfl_make(sh[0], sl[0]);
          const long long j = j0 + jj;
          dfl t0 = {0.0f, 0.0f}, t1 = {0.0f, 0.0f};
          if (MODE == M_ADAT) {
            t0 = dfl_mul(cv_df(stage, L, 0, jj), dot);
          } else if (MODE == M_RESID) {
            const dfl x = cv_df(stage, L, 0, jj);
            const dfl s = cv_df(stage, L, 1, jj);
            const dfl c = cv_df(stage, L, 2, jj);
            const dfl rd = dfl_sub(dfl_add(dot, s), c);
            const dfl d2 = dfl_div(x, s);
            a.out_df[0][j] = make_float2(rd.h, rd.l);
            a.out_df[1][j] = make_float2(d2.h, d2.l);
            t0 = x;
            const dfl xc = dfl_sub(x, dfl_div(smu, s));
            t1 = a.feasible ? xc : dfl_sub(xc, dfl_mul(d2, rd));
          } else if (MODE == M_DIR) {
            const dfl x = cv_df(stage, L, 0, jj);
            const dfl s = cv_df(stage, L, 1, jj);
            const dfl v = cv_df(stage, L, 2, jj);
            const dfl rd = a.feasible ? dfl{0.0f, 0.0f} : cv_df(stage, L, 3, jj);
            const dfl ds = dfl_neg(dfl_add(rd, dot));
            // dx = -x + (sigma mu - x ds - v) / s
            const dfl num = dfl_sub(dfl_sub(smu, dfl_mul(x, ds)), v);
            const dfl dx = dfl_sub(dfl_div(num, s), x);
            a.out_df[0][j] = make_float2(dx.h, dx.l);
            a.out_df[1][j] = make_float2(ds.h, ds.l);
          }
          t0h = t0.h;
          t0l = t0.l;
          t1h = t1.h;
          t1l = t1.l;
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
  // one accumulated output (M_ADAT) keeps v as pairs in registers: 12 consumer
  // warps so that its 128 registers per thread fit the register file
  return df_nacc<MODE>() == 2 ? (elems <= 4 ? 16 : 8)
                              : (elems <= 16 ? (df_nacc<MODE>() == 1 ? 12 : 16) : 8);
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
    cudaError_t e = ensure_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    e = launch_maybe_pdl(k, dim3(grid), dim3((CW + 1) * 32), (size_t)smem, st, a.pdl != 0, a);
    if (e != cudaSuccess) return e;
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
