// Device helpers shared by the column-streaming kernels: the bulk-copy tile
// producer, per-column vector access, the two-level deterministic reduction
// of per-CTA partials and the mode-specific epilogues on m-vectors.
#pragma once

#include "common.cuh"
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
  bulk_g2s(st, static_cast<const char*>(a.A) + (size_t)j0 * a.lda * sizeof(TA), abytes,
           &bars[stage]);
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
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < kGroup; ++q) s += (double)v[q];
      a.gpart[((size_t)grp * 2 + k) * a.lda + i] = s;
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
  auto acc_row = [&](int k, int i) -> double {
    double s = 0.0;
    for (int g = 0; g < ngroups; ++g) s += __ldcg(a.gpart + ((size_t)g * 2 + k) * a.lda + i);
    return s;
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
      double pq = 0.0;
      for (int i = tid; i < a.m; i += blockDim.x) {
        const double q = acc_row(0, i);
        a.out_m0[i] = q;
        pq += a.pcg_p[i] * q;
      }
      pq = block_sum(pq, red);
      const double alpha = a.sc->rho / pq;
      if (!(pq > 0.0) || !isfinite(alpha)) {
        if (tid == 0) atomicExch(a.err, ERR_NUMERICAL);
        return;
      }
      for (int i = tid; i < a.m; i += blockDim.x) {
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
