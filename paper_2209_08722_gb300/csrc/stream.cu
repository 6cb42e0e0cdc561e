// Column-streaming kernels over a dense column-major A: the fused
// A diag(d2) A^T v product and the FP64 passes of the outer iteration.
// See stream.cuh for the design.
#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "stream.cuh"
#include "stream_dev.cuh"

namespace lpk {

// ---------------------------------------------------------------------------
// k_stream: phase 1 per-column scalars (warp per column), phase 2 row-owned
// accumulation.  MAXRPT = row vectors per thread (compile-time maximum).
// ---------------------------------------------------------------------------
template <typename TA, typename TC, int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_stream(const StreamArgs a) {
  constexpr int VEC = VecOf<TA>::N;
  constexpr int MAXRPT = 4;
  constexpr int NACC = (MODE == M_RESID) ? 2 : ((MODE == M_ADAT || MODE == M_AX) ? 1 : 0);
  constexpr bool DOT = (MODE != M_AX);
  extern __shared__ __align__(128) char smem[];
  const SmemLayout L = make_layout(a.lda, (int)sizeof(TA), a.nb, a.stages, (int)sizeof(TC));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  TC* v_s = reinterpret_cast<TC*>(smem + L.v_off);
  double* t_s = reinterpret_cast<double*>(smem + L.t_off);
  double* red = reinterpret_cast<double*>(smem + L.red_off);
  __shared__ int s_flag;
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RV = a.lda / VEC;
  const int S = a.stages;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const double sigma_mu = a.sigma * a.sc->mu;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  if (DOT)
    for (int i = tid; i < a.lda; i += blockDim.x) v_s[i] = (i < a.m) ? (TC)a.vin[i] : (TC)0;
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < my_tiles && i < S; ++i)
      issue_tile<TA>(a, L, smem, bars, i, (int)blockIdx.x + i * (int)gridDim.x);

  // phase-2 thread mapping
  int groups, rpt, g, rv0;
  if (RV >= kThreads) {
    groups = 1;
    rpt = (RV + kThreads - 1) / kThreads;
    g = 0;
    rv0 = tid;
  } else {
    groups = kThreads / RV;
    rpt = 1;
    g = tid / RV;
    rv0 = tid % RV;
  }
  const bool p2_active = (g < groups);

  TC acc0[MAXRPT][VEC], acc1[MAXRPT][VEC];
#pragma unroll
  for (int q = 0; q < MAXRPT; ++q)
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc0[q][e] = acc1[q][e] = (TC)0;
  double cred0 = 0.0, cred1 = 0.0;  // column reductions (lane 0 of each warp)

  int consumed = 0;
  bool aborted = false;
  for (int i = 0; i < my_tiles; ++i) {
    const int st = i % S;
    const bool ok = mbar_wait(&bars[st], (uint32_t)((i / S) & 1), a.err);
    if (!__syncthreads_and(ok)) {
      aborted = true;
      break;
    }
    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
    const long long j0 = (long long)tile * a.nb;
    const int ncols = (int)min((long long)a.nb, a.n - j0);
    const char* stage = smem + (size_t)st * L.stage_bytes;
    const TA* At = reinterpret_cast<const TA*>(stage);

    // ---- phase 1: per-column scalars ----
    for (int jj = warp; jj < ncols; jj += kWarps) {
      double dot = 0.0;
      if (DOT) {
        TC d = (TC)0;
        const TA* col = At + (size_t)jj * a.lda;
        for (int rv = lane; rv < RV; rv += 32) {
          TC av[VEC];
          ld16<TC>(col + rv * VEC, av);
#pragma unroll
          for (int e = 0; e < VEC; ++e) d += av[e] * v_s[rv * VEC + e];
        }
        dot = (double)warp_sum(d);
      }
      if (lane == 0) {
        const long long j = j0 + jj;
        double t0 = 0.0, t1 = 0.0;
        if (MODE == M_ADAT) {
          t0 = cv_at(stage, L, a, 0, jj) * dot;
        } else if (MODE == M_AX) {
          t0 = cv_at(stage, L, a, 0, jj);
        } else if (MODE == M_ATY) {
          a.out_col[0][j] = dot;
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
        t_s[jj] = t0;
        t_s[a.nb + jj] = t1;
      }
    }
    if (NACC > 0) {
      __syncthreads();
      // ---- phase 2: acc += A_tile * t ----
      if (p2_active) {
        for (int jj = g; jj < ncols; jj += groups) {
          const TC t0 = (TC)t_s[jj];
          const TC t1 = (TC)t_s[a.nb + jj];
          const TA* col = At + (size_t)jj * a.lda;
#pragma unroll
          for (int q = 0; q < MAXRPT; ++q) {
            const int rv = rv0 + q * kThreads;
            if (q < rpt && rv < RV) {
              TC av[VEC];
              ld16<TC>(col + rv * VEC, av);
#pragma unroll
              for (int e = 0; e < VEC; ++e) {
                acc0[q][e] += av[e] * t0;
                if (NACC > 1) acc1[q][e] += av[e] * t1;
              }
            }
          }
        }
      }
    }
    __syncthreads();
    consumed = i + 1;
    if (tid == 0 && i + S < my_tiles) {
      fence_proxy_async_smem();
      issue_tile<TA>(a, L, smem, bars, st, (int)blockIdx.x + (i + S) * (int)gridDim.x);
    }
  }
  if (aborted && tid == 0) drain_stages<TA>(bars, consumed, my_tiles, S, a.err);
  __syncthreads();

  // ---- per-CTA partials ----
  if (NACC > 0) {
    // combine the column groups through shared memory (stage area is free now)
    TC* buf = reinterpret_cast<TC*>(smem);
    for (int k = 0; k < NACC; ++k) {
      if (p2_active) {
#pragma unroll
        for (int q = 0; q < MAXRPT; ++q) {
          const int rv = rv0 + q * kThreads;
          if (q < rpt && rv < RV)
#pragma unroll
            for (int e = 0; e < VEC; ++e)
              buf[(size_t)g * a.lda + rv * VEC + e] = (k == 0) ? acc0[q][e] : acc1[q][e];
        }
      }
      __syncthreads();
      TC* part = static_cast<TC*>(a.partials) + (size_t)blockIdx.x * 2 * a.lda + (size_t)k * a.lda;
      for (int i = tid; i < a.lda; i += blockDim.x) {
        TC s = (TC)0;
        for (int gg = 0; gg < groups; ++gg) s += buf[(size_t)gg * a.lda + i];
        part[i] = aborted ? (TC)0 : s;
      }
      __syncthreads();
    }
  }
  if (a.red_partials) {
    const double r0 = block_sum(lane == 0 ? cred0 : 0.0, red);
    const double r1 = block_sum(lane == 0 ? cred1 : 0.0, red);
    if (tid == 0) {
      a.red_partials[2 * blockIdx.x] = r0;
      a.red_partials[2 * blockIdx.x + 1] = r1;
    }
  }
  if (a.epilogue == E_NONE) return;
  if (tree_reduce<TC>(a, NACC, &s_flag)) stream_epilogue<TC>(a, NACC, red);
}

// ---------------------------------------------------------------------------
// k_adat_fused: u = A diag(d2) A^T v in FP32 (the product inside every CG
// step).  Warp-specialised: warp kConsumerWarps is the producer (one lane
// issues the bulk copies of tile i into stage i % S once the consumers have
// released it on empty[i % S]); the kConsumerWarps consumer warps each take
// whole columns of a tile (column jj goes to warp jj % kConsumerWarps): load
// the column slice from shared memory into registers once, form d2_j (a_j^T v)
// (four independent partial sums, then a warp reduction) and accumulate
// a_j t_j into per-lane registers covering all rows.  No CTA-wide barrier
// inside the stream.  VPL = 16-byte vectors per lane per column.
// ---------------------------------------------------------------------------
template <typename TA, int VPL>
__global__ void __launch_bounds__(kFusedThreads, 1) k_adat_fused(const StreamArgs a) {
  constexpr int VEC = VecOf<TA>::N;
  constexpr bool VREG = (VPL * VEC <= 32);
  extern __shared__ __align__(128) char smem[];
  const SmemLayout L = make_layout(a.lda, (int)sizeof(TA), a.nb, a.stages, 4);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* empty = full + a.stages;
  float* v_s = reinterpret_cast<float*>(smem + L.v_off);
  double* red = reinterpret_cast<double*>(smem + L.red_off);
  __shared__ int s_flag;
  pdl_wait();
  pdl_trigger();
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RV = a.lda / VEC;
  const int S = a.stages;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kConsumerWarps);
    }
    fence_mbar_init();
  }
  for (int i = tid; i < a.lda; i += blockDim.x) v_s[i] = (i < a.m) ? (float)a.vin[i] : 0.0f;
  __syncthreads();

  float acc[VPL][VEC];
#pragma unroll
  for (int c = 0; c < VPL; ++c)
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[c][e] = 0.0f;
  bool aborted = false;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
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
      if (aborted || *a.err != ERR_NONE) {
        // make sure no copy is still landing in shared memory before exit
        for (int j = (issued > S ? issued - S : 0); j < issued; ++j)
          mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), a.err);
      }
    }
  } else {
    // ---------------- consumers ----------------
    float vr[VREG ? VPL : 1][VREG ? VEC : 1];
    if (VREG) {
#pragma unroll
      for (int c = 0; c < VPL; ++c)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const int rv = c * 32 + lane;
          vr[c][e] = (rv < RV) ? v_s[rv * VEC + e] : 0.0f;
        }
    }
    for (int i = 0; i < my_tiles; ++i) {
      const int st = i % S;
      if (!mbar_wait(&full[st], (uint32_t)((i / S) & 1), a.err)) {
        aborted = true;
        break;
      }
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const long long j0 = (long long)tile * a.nb;
      const int ncols = (int)min((long long)a.nb, a.n - j0);
      const char* stage = smem + (size_t)st * L.stage_bytes;
      const TA* At = reinterpret_cast<const TA*>(stage);
      const float* d2t = reinterpret_cast<const float*>(stage + L.cv_off[0]);
      for (int jj = warp; jj < ncols; jj += kConsumerWarps) {
        const TA* col = At + (size_t)jj * a.lda;
        float av[VPL][VEC];
        float dp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < VPL; ++c) {
          const int rv = c * 32 + lane;
          if (rv < RV) {
            ld16<float>(col + rv * VEC, av[c]);
          } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) av[c][e] = 0.0f;
          }
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float vv = VREG ? vr[VREG ? c : 0][VREG ? e : 0]
                                  : ((rv < RV) ? v_s[rv * VEC + e] : 0.0f);
            dp[(c * VEC + e) & 3] = fmaf(av[c][e], vv, dp[(c * VEC + e) & 3]);
          }
        }
        float d = (dp[0] + dp[1]) + (dp[2] + dp[3]);
        d = warp_sum(d);
        const float t = d2t[jj] * d;
#pragma unroll
        for (int c = 0; c < VPL; ++c)
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[c][e] = fmaf(av[c][e], t, acc[c][e]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  aborted = __syncthreads_or(aborted) != 0;
  // cross-warp reduction through shared memory: buf[consumer warp][lda]
  float* buf = reinterpret_cast<float*>(smem);
  if (warp < kConsumerWarps) {
#pragma unroll
    for (int c = 0; c < VPL; ++c) {
      const int rv = c * 32 + lane;
      if (rv < RV)
#pragma unroll
        for (int e = 0; e < VEC; ++e) buf[(size_t)warp * a.lda + rv * VEC + e] = acc[c][e];
    }
  }
  __syncthreads();
  float* part = static_cast<float*>(a.partials) + (size_t)blockIdx.x * 2 * a.lda;
  for (int r = tid; r < a.lda; r += blockDim.x) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kConsumerWarps; ++w) s += buf[(size_t)w * a.lda + r];
    part[r] = aborted ? 0.0f : s;
  }
  if (a.epilogue == E_NONE) return;
  if (tree_reduce<float>(a, 1, &s_flag)) stream_epilogue<float>(a, 1, red);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

template <typename TA, typename TC, int MODE>
cudaError_t launch_stream_t(const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  auto k = k_stream<TA, TC, MODE>;
  cudaError_t e = ensure_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename TA, int VPL>
cudaError_t launch_fused_t(const StreamArgs& a, int grid, int smem, cudaStream_t st, bool pdl) {
  auto k = k_adat_fused<TA, VPL>;
  cudaError_t e = ensure_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  e = launch_maybe_pdl(k, dim3(grid), dim3(kFusedThreads), (size_t)smem, st, pdl, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename TA, typename TC>
cudaError_t dispatch_mode(int mode, const StreamArgs& a, int grid, int smem, cudaStream_t st) {
  switch (mode) {
    case M_ADAT: return launch_stream_t<TA, TC, M_ADAT>(a, grid, smem, st);
    case M_AX: return launch_stream_t<TA, TC, M_AX>(a, grid, smem, st);
    case M_RESID: return launch_stream_t<TA, TC, M_RESID>(a, grid, smem, st);
    case M_DIR: return launch_stream_t<TA, TC, M_DIR>(a, grid, smem, st);
    case M_ATY: return launch_stream_t<TA, TC, M_ATY>(a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

template <typename TA>
cudaError_t dispatch_fused(int vpl, const StreamArgs& a, int grid, int smem, cudaStream_t st, bool pdl) {
  switch (vpl) {
    case 1: return launch_fused_t<TA, 1>(a, grid, smem, st, pdl);
    case 2: return launch_fused_t<TA, 2>(a, grid, smem, st, pdl);
    case 4: return launch_fused_t<TA, 4>(a, grid, smem, st, pdl);
    case 8: return launch_fused_t<TA, 8>(a, grid, smem, st, pdl);
    case 16: return launch_fused_t<TA, 16>(a, grid, smem, st, pdl);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

StreamPlan make_stream_plan(int m, long long n, int lda, int esz, int num_sms, int tc_bytes) {
  return make_stream_plan_ex(m, n, lda, esz, num_sms, tc_bytes, 32 * 1024, kMaxStages);
}

// tiles of about target_bytes of A (4 to 64 columns, a multiple of 4), and as
// many stages (at most max_stages) as fit the shared-memory budget
StreamPlan make_stream_plan_ex(int m, long long n, int lda, int esz, int num_sms, int tc_bytes, int target,
                               int max_stages) {
  StreamPlan p;
  const int col_bytes = lda * esz;
  int nb = target / col_bytes;
  nb = std::max(4, std::min(64, nb));
  nb = nb / 4 * 4;
  p.nb = nb;
  p.ntiles = (int)((n + nb - 1) / nb);
  const int budget = 220 * 1024;
  int stages = std::max(2, std::min(kMaxStages, max_stages));
  for (; stages >= 2; --stages) {
    SmemLayout L = make_layout(lda, esz, nb, stages, 8);
    // the end-of-kernel reduction buffer reuses the stage area
    const int redbuf = std::max(kConsumerWarps * lda * 4, kThreads / std::max(1, lda / (16 / esz)) * lda * 8);
    if (L.total <= budget && stages * L.stage_bytes >= redbuf) break;
  }
  if (stages < 2) stages = 2;
  p.stages = stages;
  p.grid = std::max(1, std::min(std::min(p.ntiles, num_sms), kGroup * kMaxGroups));
  p.smem = make_layout(lda, esz, nb, stages, tc_bytes).total;
  p.smem8 = make_layout(lda, esz, nb, stages, 8).total;
  p.ok = (p.smem8 <= 227 * 1024);
  (void)m;
  return p;
}

int fused_vpl(int lda, int esz) {
  const int vec = 16 / esz;
  const int rv = lda / vec;
  const int need = (rv + 31) / 32;
  for (int v : {1, 2, 4, 8, 16})
    if (need <= v) return v;
  return 0;
}

cudaError_t launch_stream(int dtype, bool fp64_acc, int mode, const StreamArgs& a,
                          const StreamPlan& p, cudaStream_t st) {
  const int smem = fp64_acc ? p.smem8 : p.smem;
  if (dtype == 0) return dispatch_mode<double, double>(mode, a, p.grid, p.smem8, st);
  if (dtype == 1) {
    if (fp64_acc) return dispatch_mode<float, double>(mode, a, p.grid, smem, st);
    return dispatch_mode<float, float>(mode, a, p.grid, smem, st);
  }
  if (fp64_acc) return dispatch_mode<bf16raw, double>(mode, a, p.grid, smem, st);
  return dispatch_mode<bf16raw, float>(mode, a, p.grid, smem, st);
}

cudaError_t launch_adat_fused(int dtype, const StreamArgs& a, const StreamPlan& p,
                              cudaStream_t st, bool pdl) {
  const int esz = dtype == 1 ? 4 : 2;
  const int vpl = fused_vpl(a.lda, esz);
  if (vpl == 0) return cudaErrorInvalidValue;
  if (dtype == 1) return dispatch_fused<float>(vpl, a, p.grid, p.smem, st, pdl);
  if (dtype == 2) return dispatch_fused<bf16raw>(vpl, a, p.grid, p.smem, st, pdl);
  return cudaErrorInvalidValue;
}

}  // namespace lpk
