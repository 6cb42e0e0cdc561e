// Device helpers shared by the column-streaming kernels: the bulk-copy tile
// producer, per-column vector access, the two-level deterministic reduction
// of per-CTA partials and the mode-specific epilogues on m-vectors.
#pragma once

#include "common.cuh"
#include "df.cuh"
#include "stream.cuh"

namespace lpk {

// ---------------------------------------------------------------------------
// tile producer (one thread)
// ---------------------------------------------------------------------------
template <typename TA>
__device__ __forceinline__ void issue_tile(const StreamArgs& a, const SmemLayout& L, char* smem,
                                           uint64_t* bars, int stage, int tile) {
  const long long j0 = (long long)tile * a.nb;
  const int ncols = (int)min((long long)a.nb, a.n - j0);
  char* st = smem + (size_t)stage * L.stage_bytes;
  const uint32_t abytes = (uint32_t)ncols * (uint32_t)a.lda * (uint32_t)sizeof(TA);
  uint32_t total = abytes;
  uint32_t cvb[kMaxColVecs];
#pragma unroll
  for (int q = 0; q < kMaxColVecs; ++q) {
    cvb[q] = (q < a.ncv) ? (uint32_t)align_up_i(ncols * a.cv_esz[q], 16) : 0u;
    total += cvb[q];
  }
  mbar_arrive_expect_tx(&bars[stage], total);
  bulk_g2s_stream(st, static_cast<const char*>(a.A) + (size_t)j0 * a.lda * sizeof(TA), abytes, &bars[stage]);
#pragma unroll
  for (int q = 0; q < kMaxColVecs; ++q)
    if (q < a.ncv)
      bulk_g2s(st + L.cv_off[q], static_cast<const char*>(a.cv[q]) + (size_t)j0 * a.cv_esz[q],
               cvb[q], &bars[stage]);
}

__device__ __forceinline__ double cv_at(const char* stage, const SmemLayout& L, const StreamArgs& a,
                                        int q, int jj) {
  const char* p = stage + L.cv_off[q];
  return a.cv_esz[q] == 8 ? reinterpret_cast<const double*>(p)[jj]
                          : (double)reinterpret_cast<const float*>(p)[jj];
}

// Waits (bounded) on every stage still holding an issued copy; used when aborting.
template <typename TA>
__device__ void drain_stages(uint64_t* bars, int consumed, int my_tiles, int S, int* err) {
  for (int i = consumed; i < my_tiles && i < consumed + S; ++i)
    mbar_wait(&bars[i % S], (i / S) & 1, err);
}

// ---------------------------------------------------------------------------
// epilogue run by the last CTA: FP64 reduction of the per-CTA partials in a
// fixed order, then the mode-specific vector work on m-vectors.
// ---------------------------------------------------------------------------
// Two-level deterministic reduction of the per-CTA partial vectors.  CTAs form
// groups of kGroup consecutive blocks; the last CTA of a group to finish (group
// ticket) sums that group's partials in FP64 in block order into gpart[group],
// then takes the global ticket; the last group reducer returns true and its
// CTA then holds every group sum.  Group sums overlap the other CTAs' streaming.
template <typename TC>
__device__ bool tree_reduce(const StreamArgs& a, int nacc, int* s_flag) {
  const int G = gridDim.x;
  const int ngroups = (G + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup;
  const int b0 = grp * kGroup;
  const int gsize = min(kGroup, G - b0);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(a.gtickets + grp, 1u);
    const bool last = (t == (unsigned)gsize - 1u);
    if (last) a.gtickets[grp] = 0u;
    *s_flag = last ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag == 0) return false;
  __threadfence();
  const TC* part = static_cast<const TC*>(a.partials);
  const size_t pstride = (size_t)2 * a.lda;
  for (int k = 0; k < nacc; ++k)
    for (int i = threadIdx.x; i < a.lda; i += blockDim.x) {
      TC v[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q)
        v[q] = (q < gsize) ? __ldcg(part + (size_t)(b0 + q) * pstride + (size_t)k * a.lda + i) : (TC)0;
      if constexpr (sizeof(TC) == 4) {
        // FP32 partials: the group sum as an FP32 pair (FP32 pipe; an FP64
        // warp instruction costs GB300's FP64 unit about 16 cycles)
        float sh = 0.0f, sl = 0.0f;
#pragma unroll
        for (int q = 0; q < kGroup; ++q) df_add(sh, sl, (float)v[q], 0.0f);
        df_renorm(sh, sl);
        reinterpret_cast<float2*>(a.gpart)[((size_t)grp * 2 + k) * a.lda + i] = make_float2(sh, sl);
      } else {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kGroup; ++q) s += (double)v[q];
        a.gpart[((size_t)grp * 2 + k) * a.lda + i] = s;
      }
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(a.gtickets + kMaxGroups, 1u);
    const bool last = (t == (unsigned)ngroups - 1u);
    if (last) a.gtickets[kMaxGroups] = 0u;
    *s_flag = last ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag == 0) return false;
  __threadfence();
  return true;
}

template <typename TC>
__device__ void stream_epilogue(const StreamArgs& a, int nacc, double* red) {
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int ngroups = (G + kGroup - 1) / kGroup;
  if (*a.err != ERR_NONE) return;
  // sum of row i over the group sums, in group order; the loads are issued
  // eight at a time so that their L2 latencies overlap
  auto acc_row = [&](int k, int i) -> double {
    const size_t gs = (size_t)2 * a.lda;
    if constexpr (sizeof(TC) == 4) {
      // group sums held as FP32 pairs: summed as pairs, one conversion at the end
      const float2* base = reinterpret_cast<const float2*>(a.gpart) + (size_t)k * a.lda + i;
      float sh = 0.0f, sl = 0.0f;
      for (int g0 = 0; g0 < ngroups; g0 += 8) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          v[q] = (g0 + q < ngroups) ? __ldcg(base + (size_t)(g0 + q) * gs) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 8; ++q) df_add(sh, sl, v[q].x, v[q].y);
      }
      return (double)sh + (double)sl;
    } else {
      const double* base = a.gpart + (size_t)k * a.lda + i;
      double s = 0.0;
      for (int g0 = 0; g0 < ngroups; g0 += 8) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (g0 + q < ngroups) ? __ldcg(base + (size_t)(g0 + q) * gs) : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (g0 + q < ngroups) s += v[q];
      }
      return s;
    }
  };
  // column reductions (two FP64 sums over columns), block-parallel in a fixed order
  double cr0 = 0.0, cr1 = 0.0;
  if (a.red_partials) {
    double t0 = 0.0, t1 = 0.0;
    for (int b = tid; b < G; b += blockDim.x) {
      t0 += __ldcg(a.red_partials + 2 * b);
      t1 += __ldcg(a.red_partials + 2 * b + 1);
    }
    cr0 = block_sum(t0, red);
    cr1 = block_sum(t1, red);
  }
  switch (a.epilogue) {
    case E_PLAIN:
      for (int i = tid; i < a.m; i += blockDim.x) {
        a.out_m0[i] = acc_row(0, i);
        if (nacc > 1) a.out_m1[i] = acc_row(1, i);
      }
      break;
    case E_TRUE_RES:
      for (int i = tid; i < a.m; i += blockDim.x) a.pcg_r[i] = a.bvec[i] - acc_row(0, i);
      break;
    case E_PCG_A: {
      // the first kRows rows of each thread stay in registers (q, p, dy, r all
      // loaded before the reduction of p^T q); rows beyond are re-read
      constexpr int kRows = 4;
      double qv[kRows], pv[kRows], dv[kRows], rv[kRows];
      double pq = 0.0;
#pragma unroll
      for (int c = 0; c < kRows; ++c) {
        const int i = tid + c * (int)blockDim.x;
        if (i < a.m) {
          pv[c] = a.pcg_p[i];
          dv[c] = a.pcg_dy[i];
          rv[c] = a.pcg_r[i];
          qv[c] = acc_row(0, i);
          a.out_m0[i] = qv[c];
          pq += pv[c] * qv[c];
        }
      }
      for (int i = tid + kRows * (int)blockDim.x; i < a.m; i += blockDim.x) {
        const double q = acc_row(0, i);
        a.out_m0[i] = q;
        pq += a.pcg_p[i] * q;
      }
      // p^T q: each thread's FP64 partial as an FP32 pair, reduced on the FP32
      // pipe; alpha = rho / p^T q once, in thread 0, and broadcast
      {
        float ph = (float)pq;
        float pl = (float)(pq - (double)ph);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, ph, off);
          const float ol = __shfl_xor_sync(0xffffffffu, pl, off);
          df_add(ph, pl, oh, ol);
        }
        float2* redf = reinterpret_cast<float2*>(red);
        const int nw = (int)(blockDim.x + 31) / 32;
        __syncthreads();
        if ((tid & 31) == 0) redf[tid >> 5] = make_float2(ph, pl);
        __syncthreads();
        if (tid == 0) {
          float sh = 0.0f, sl = 0.0f;
          for (int w = 0; w < nw; ++w) df_add(sh, sl, redf[w].x, redf[w].y);
          const double pqs = (double)sh + (double)sl;
          const double al = a.sc->rho / pqs;
          const bool bad = !(pqs > 0.0) || !isfinite(al);
          if (bad) atomicExch(a.err, ERR_NUMERICAL);
          red[32] = al;
          red[33] = pqs;
          red[34] = bad ? 1.0 : 0.0;
        }
        __syncthreads();
        pq = red[33];
      }
      const double alpha = red[32];
      if (red[34] != 0.0) return;  // breakdown (p^T q <= 0 or non-finite), flagged above
#pragma unroll
      for (int c = 0; c < kRows; ++c) {
        const int i = tid + c * (int)blockDim.x;
        if (i < a.m) {
          a.pcg_dy[i] = dv[c] + alpha * pv[c];
          a.pcg_r[i] = rv[c] - alpha * qv[c];
        }
      }
      for (int i = tid + kRows * (int)blockDim.x; i < a.m; i += blockDim.x) {
        a.pcg_dy[i] += alpha * a.pcg_p[i];
        a.pcg_r[i] -= alpha * a.out_m0[i];
      }
      if (tid == 0) {
        a.sc->pq = pq;
        const int it = a.sc->inner_iters;
        if (a.coef && it < 1024) a.coef[2 * it] = alpha;
      }
      break;
    }
    case E_CHEB:
      for (int i = tid; i < a.m; i += blockDim.x) a.pcg_r[i] -= acc_row(0, i);
      break;
    case E_RESID: {
      double rp2 = 0.0, by = 0.0;
      for (int i = tid; i < a.m; i += blockDim.x) {
        const double rp = acc_row(0, i) - a.bvec[i];
        const double ap = acc_row(1, i);
        a.out_m0[i] = rp;
        a.out_m1[i] = a.feasible ? ap : ap - rp;
        rp2 += rp * rp;
        by += a.bvec[i] * a.vin[i];
      }
      rp2 = block_sum(rp2, red);
      by = block_sum(by, red);
      if (tid == 0) {
        a.sc->rp2 = rp2;
        a.sc->by = by;
        a.sc->rd2 = cr0;
        a.sc->cx = cr1;
      }
      break;
    }
    case E_DIR:
      if (tid == 0) {
        a.sc->c1 = cr0 / (double)a.n;
        a.sc->c2 = cr1 / (double)a.n;
      }
      break;
    default:
      break;
  }
}

}  // namespace lpk
