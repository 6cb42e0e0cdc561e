// Explicit preconditioner Q^{-1} = ((ADW)(ADW)^T)^{-1} (Algorithm 1 step 2;
// eq. precond uses Q^{-1} in every inner iteration) by a blocked symmetric
// Gauss-Jordan elimination (the sweep operator of Beaton/Goodnight) in
// double-float arithmetic.
//
// Sweeping a symmetric matrix on a pivot block K maps
//     A_KK -> -A_KK^{-1},   A_IK -> A_IK A_KK^{-1},   A_KJ -> A_KK^{-1} A_KJ,
//     A_IJ -> A_IJ - A_IK A_KK^{-1} A_KJ                      (I, J outside K),
// and sweeping every pivot block in turn leaves -A^{-1}.  Without pivoting
// this is stable for symmetric positive definite A (its pivots are the
// squares of the Cholesky diagonal, which also give the rank check).
//
// GB300 runs FP64 at a small fraction of the FP32 rate, and the factor of an
// m x m matrix with m in the hundreds is latency-bound in library code, so:
//   * the matrix is prescaled by a power of two (max diagonal -> [1, 2)) and
//     held as FP32 pairs (relative accuracy ~2^-46 per operation);
//   * each of the m/32 pivot steps is two launches: one CTA of 32 x 32 threads
//     sweeps the 32 x 32 pivot block (the step's serial chain of 32 pivots,
//     one element per thread), then one launch over all 32 x 32 tiles writes
//     the next iterate from it; two buffers alternate, so no tile is read after
//     it is overwritten.
#include "internal.h"
#include "df.cuh"

namespace lpk {

namespace {
constexpr int SB = 32;          // pivot block = tile
constexpr int SW_THREADS = 256; // 8 x 32 threads, 4 outputs each

// (ah + al)(bh + bl) as a normalised pair
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  ph = __fadd_rn(p, e);
  pl = __fsub_rn(e, __fsub_rn(ph, p));
}

// (sh, sl) += (ah + al)(bh + bl)
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s, q;
  two_sum(sh, p, s, q);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(q, e));
}

// 1 / (dh + dl): FP32 reciprocal plus one Newton correction in double-float
__device__ __forceinline__ void df_recip(float dh, float dl, float& rh, float& rl) {
  const float r0 = __frcp_rn(dh);
  const float p = __fmul_rn(dh, r0);
  const float pe = fmaf(dh, r0, -p);
  // e = 1 - (dh + dl) r0, where 1 - p is exact (p is within an ulp of 1)
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(dl, r0));
  const float c = __fmul_rn(r0, e);
  rh = __fadd_rn(r0, c);
  rl = __fsub_rn(c, __fsub_rn(rh, r0));
}
}  // namespace

// A0 = 2^-e G (symmetric, both triangles, padded to mp with the identity) as
// a pair of FP32 arrays; G holds the upper triangle of a column-major m x m.
// Every CTA first finds the max diagonal (m loads) to pick e.
__global__ void __launch_bounds__(256) k_sweep_init(const double* __restrict__ g, int m, int mp,
                                                    float* __restrict__ ah, float* __restrict__ al,
                                                    double* __restrict__ scale_out) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) mx = fmax(mx, fabs(g[(size_t)i * m + i]));
  mx = -block_min(-mx, red);
  const int e = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = ldexp(1.0, e);
  const long long total = (long long)mp * mp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / mp), j = (int)(t % mp);
    double v;
    if (i < m && j < m) v = ldexp(i <= j ? g[(size_t)j * m + i] : g[(size_t)i * m + j], -e);
    else v = i == j ? 1.0 : 0.0;
    const float hi = (float)v;
    ah[t] = hi;
    al[t] = (float)(v - (double)hi);
  }
}

// The pivot block of step K swept on its 32 pivots, once: P -> -P^{-1} into
// (qh, ql), and the pivots (the squares of the Cholesky diagonal) into piv.
// One CTA of SB x SB threads, thread (a, b) owning entry (a, b); per pivot t
// every thread reads d = P_tt, P_at and P_bt, then writes its new entry
// (a == t or b == t: the scaled column or -1/d; otherwise P_ab - (P_at/d) P_bt).
__global__ void __launch_bounds__(SB* SB) k_sweep_pivot(const float* __restrict__ sh_, const float* __restrict__ sl_,
                                                       int mp, int K, float* __restrict__ qh,
                                                       float* __restrict__ ql, float* __restrict__ piv) {
  __shared__ float Ph[SB][SB + 1], Pl[SB][SB + 1];
  const int a = threadIdx.x / SB, b = threadIdx.x % SB;
  const int k0 = K * SB;
  {
    const size_t src = (size_t)(k0 + a) * mp + k0 + b;
    Ph[a][b] = sh_[src];
    Pl[a][b] = sl_[src];
  }
  __syncthreads();
  for (int t = 0; t < SB; ++t) {
    const float dh = Ph[t][t], dl = Pl[t][t];
    const float ah = Ph[a][t], al = Pl[a][t];
    const float bh = Ph[b][t], bl = Pl[b][t];
    float h = Ph[a][b], l = Pl[a][b];
    __syncthreads();  // every read of this pivot's iterate is done
    float rh, rl;
    df_recip(dh, dl, rh, rl);
    if (threadIdx.x == 0 && piv) piv[k0 + t] = dh;
    if (a == t && b == t) {
      h = -rh;
      l = -rl;
    } else if (a == t) {
      df_mul(bh, bl, rh, rl, h, l);  // P_bt / d
    } else {
      float wh, wl;
      df_mul(ah, al, rh, rl, wh, wl);  // P_at / d
      if (b == t) {
        h = wh;
        l = wl;
      } else {
        df_mac(-wh, -wl, bh, bl, h, l);
        df_renorm(h, l);
      }
    }
    Ph[a][b] = h;
    Pl[a][b] = l;
    __syncthreads();
  }
  qh[a * SB + b] = Ph[a][b];
  ql[a * SB + b] = Pl[a][b];
}

// one pivot step K: src -> dst for every 32 x 32 tile (I, J); the swept pivot
// block -P^{-1} comes from k_sweep_pivot
__global__ void __launch_bounds__(SW_THREADS) k_sweep_step(const float* __restrict__ sh_, const float* __restrict__ sl_,
                                                           float* __restrict__ dh_, float* __restrict__ dl_,
                                                           int mp, int K, const float* __restrict__ qh,
                                                           const float* __restrict__ ql) {
  __shared__ float Ph[SB][SB + 1], Pl[SB][SB + 1];  // pivot block, swept in place -> -P^{-1}
  __shared__ float Ch[SB][SB + 1], Cl[SB][SB + 1];  // panel rows of the other block: A_{J,K}
  __shared__ float Th[SB][SB + 1], Tl[SB][SB + 1];  // A_{X,K} (-P^{-1})... see below
  const int nt = mp / SB;
  const int I = blockIdx.x % nt, J = blockIdx.x / nt;
  const int k0 = K * SB;
  const int tid = threadIdx.x;
  const int r = tid >> 3, c4 = (tid & 7) * 4;  // this thread's outputs: row r, columns c4..c4+3

  // ---- load the swept pivot block -P^{-1} ----
  for (int e = tid; e < SB * SB; e += SW_THREADS) {
    const int a = e / SB, b = e % SB;
    Ph[a][b] = qh[e];
    Pl[a][b] = ql[e];
  }
  // ---- load the panels needed by this tile ----
  // case 1 (I != K, J != K): T <- A_{I,K}, C <- A_{J,K}; case 2 (J == K): T <- A_{I,K};
  // case 3 (I == K): T <- A_{J,K}
  const int X = (I == K) ? J : I;
  if (X != K) {
    for (int e = tid; e < SB * SB; e += SW_THREADS) {
      const int a = e / SB, b = e % SB;
      const size_t src = (size_t)(X * SB + a) * mp + k0 + b;
      Th[a][b] = sh_[src];
      Tl[a][b] = sl_[src];
    }
  }
  if (I != K && J != K) {
    for (int e = tid; e < SB * SB; e += SW_THREADS) {
      const int a = e / SB, b = e % SB;
      const size_t src = (size_t)(J * SB + a) * mp + k0 + b;
      Ch[a][b] = sh_[src];
      Cl[a][b] = sl_[src];
    }
  }
  __syncthreads();

  // ---- this thread's four outputs ----
  float oh[4], ol[4];
  if (I == K && J == K) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      oh[q] = Ph[r][c4 + q];  // -P^{-1}
      ol[q] = Pl[r][c4 + q];
    }
  } else {
    // U = A_{X,K} (-P^{-1}) = -(A_{X,K} P^{-1}) for this thread's row r
    float uh4[4], ul4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uh4[q] = 0.0f;
      ul4[q] = 0.0f;
    }
    // row r of U for all 32 columns is needed in case 1: compute the full
    // 32 x 32 U into smem first (each thread its 4 entries), then use it
    for (int b = 0; b < SB; ++b) {
      const float th = Th[r][b], tl = Tl[r][b];
#pragma unroll
      for (int q = 0; q < 4; ++q) df_mac(th, tl, Ph[b][c4 + q], Pl[b][c4 + q], uh4[q], ul4[q]);
    }
    __syncthreads();  // all reads of T done before it is overwritten with U
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      df_renorm(uh4[q], ul4[q]);
      Th[r][c4 + q] = uh4[q];
      Tl[r][c4 + q] = ul4[q];
    }
    __syncthreads();
    if (J == K) {
      // A_IK P^{-1} = -U
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        oh[q] = -Th[r][c4 + q];
        ol[q] = -Tl[r][c4 + q];
      }
    } else if (I == K) {
      // P^{-1} A_KJ = (A_JK P^{-1})^T = -U^T
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        oh[q] = -Th[c4 + q][r];
        ol[q] = -Tl[c4 + q][r];
      }
    } else {
      // A_IJ - A_IK P^{-1} A_KJ = A_IJ + U A_{J,K}^T
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const size_t src = (size_t)(I * SB + r) * mp + J * SB + c4 + q;
        oh[q] = sh_[src];
        ol[q] = sl_[src];
      }
      for (int b = 0; b < SB; ++b) {
        const float th = Th[r][b], tl = Tl[r][b];
#pragma unroll
        for (int q = 0; q < 4; ++q) df_mac(th, tl, Ch[c4 + q][b], Cl[c4 + q][b], oh[q], ol[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    df_renorm(oh[q], ol[q]);
    const size_t dst = (size_t)(I * SB + r) * mp + J * SB + c4 + q;
    dh_[dst] = oh[q];
    dl_[dst] = ol[q];
  }
}

// Q^{-1} = -2^-e A_final (FP64, m x m, both triangles) and the rank check on
// the pivots (|R_ii| = sqrt(pivot_i))
__global__ void __launch_bounds__(256) k_sweep_finish(const float* __restrict__ ah, const float* __restrict__ al,
                                                      int m, int mp, const double* __restrict__ scale,
                                                      const float* __restrict__ piv, double* __restrict__ qinv,
                                                      float2* __restrict__ qinv_df, DevScalars* sc,
                                                      double rank_tol) {
  __shared__ double red[32];
  const double s = *scale;
  if (blockIdx.x == 0) {
    double mn = INFINITY, mx = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const float p = piv[i];
      if (!(p > 0.0f) || !isfinite(p)) bad = true;
      const double d = sqrt((double)fmaxf(p, 0.0f) * s);
      mn = fmin(mn, d);
      mx = fmax(mx, d);
    }
    const int any_bad = __syncthreads_or(bad);
    mn = block_min(mn, red);
    mx = -block_min(-mx, red);
    if (threadIdx.x == 0) {
      sc->diag_min = mn;
      sc->diag_max = mx;
      sc->rank_bad = (any_bad || !(mn > rank_tol * mx) || !isfinite(mx)) ? 1 : 0;
    }
  }
  // -2^-e A as pairs: scaling by a power of two is exact in FP32 as well
  const int e = ilogb(s);
  const long long total = (long long)m * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / m), j = (int)(t % m);
    const size_t src = (size_t)i * mp + j;
    if (qinv) qinv[t] = -ldexp((double)ah[src] + (double)al[src], -e);
    if (qinv_df) qinv_df[t] = make_float2(-ldexpf(ah[src], -e), -ldexpf(al[src], -e));
  }
}

size_t sweep_scratch_floats(int m) {
  const size_t mp = (size_t)(m + SB - 1) / SB * SB;
  return 4 * mp * mp + mp + 8 + 2 * SB * SB;
}

// G: upper triangle of the column-major m x m Gram; qinv: m x m output
cudaError_t launch_sweep_inverse(const double* g, int m, float* scratch, double* qinv, float2* qinv_df,
                                 DevScalars* sc, double rank_tol, int num_sms, cudaStream_t st) {
  const int mp = (m + SB - 1) / SB * SB;
  const size_t mm = (size_t)mp * mp;
  float* a0h = scratch;
  float* a0l = scratch + mm;
  float* a1h = scratch + 2 * mm;
  float* a1l = scratch + 3 * mm;
  float* piv = scratch + 4 * mm;
  // the prescale 2^e, 8-byte aligned after the mp pivots (mp is a multiple of 32)
  double* scale_buf = reinterpret_cast<double*>(scratch + 4 * mm + mp);
  float* qh = scratch + 4 * mm + mp + 8;  // the swept pivot block of the current step
  float* ql = qh + SB * SB;
  const int g1 = (int)std::max<long long>(1, std::min<long long>(((long long)mm + 255) / 256, (long long)num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_sweep_init<<<g1, 256, 0, st>>>(g, m, mp, a0h, a0l, scale_buf);
  const int nt = mp / SB;
  for (int K = 0; K < nt; ++K) {
    const bool even = (K & 1) == 0;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_sweep_pivot<<<1, SB * SB, 0, st>>>(even ? a0h : a1h, even ? a0l : a1l, mp, K, qh, ql, piv);
    k_sweep_step<<<nt * nt, SW_THREADS, 0, st>>>(even ? a0h : a1h, even ? a0l : a1l, even ? a1h : a0h,
                                                 even ? a1l : a0l, mp, K, qh, ql);
  }
  const bool in0 = (nt & 1) == 0;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const int g2 = (int)std::max<long long>(1, std::min<long long>(((long long)m * m + 255) / 256, (long long)num_sms * 4));
  k_sweep_finish<<<g2, 256, 0, st>>>(in0 ? a0h : a1h, in0 ? a0l : a1l, m, mp, scale_buf, piv, qinv, qinv_df, sc,
                                     rank_tol);
  return cudaGetLastError();
}

}  // namespace lpk
