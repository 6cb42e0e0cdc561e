// Row-split column-streaming kernels for tall columns (large m).
//
// The warp-per-column kernels (k_adat_fused, k_stream_df) keep one column in
// registers per lane while they accumulate a_j t_j over all m rows, so their
// per-lane state grows with m: beyond 1024 rows (BF16) or 512 rows (FP32) it
// no longer fits the register file and spills.  Here the rows of a column are
// split across warps instead, so every lane owns a fixed slice of rows for the
// whole stream:
//
//   * rows come in slabs of 32 16-byte row vectors (one per lane); a warp owns
//     RPT consecutive slabs (two for the FP32 product, one for the
//     double-float passes where the rows allow), nsw warps cover a column, and
//     the 16 consumer warps form L = 16 / nsw column groups;
//   * a tile holds CPT = 4 columns per group (nb = 4 L columns, 32-64 KB),
//     streamed by one producer lane with cp.async.bulk into a ring of stages
//     (full/empty mbarriers, as in the other streaming kernels);
//   * phase 1: each warp forms its slab's partial of a_j^T v for the group's
//     four columns (v's slice held in registers), reduces it over its lanes and
//     writes it to a double-buffered shared array; one named barrier over the
//     consumer warps (which also votes on an aborted wait) publishes them;
//   * the column scalars t_j (d2_j (a_j^T v), or the residual / direction
//     formulas) are summed over the nsw partials in a fixed order by lane c of
//     every warp of the group (so all of them get identical values) and
//     broadcast by shuffles;
//   * phase 2: each lane adds a_j t_j to the accumulators of its rows, reading
//     its column slices from the stage again (shared memory is read twice per
//     element; keeping them in registers would not leave room for the
//     accumulators);
//   * the L groups' accumulators of the same rows are combined at the end and
//     go through the deterministic two-level reduction and the mode epilogues
//     shared with the other streaming kernels.
// Two arithmetics: FP32 products with FP32 accumulation (the inner-loop
// product, M_ADAT) and double-float (FP32 pairs: exact FMA products and
// TwoSum accumulation, as in stream_df.cu) for the FP64-class passes M_ADAT
// (the residual refresh), M_RESID and M_DIR.
#include <type_traits>

#include "internal.h"
#include "stream_dev.cuh"
#include "df.cuh"

namespace lpk {

namespace {

constexpr int kRowsCPT = 4;      // columns per column group per tile
constexpr int kRowsMaxStages = 8;

__host__ __device__ inline void rows_geom(int lda, int esz, int rpt, int* nsw, int* groups) {
  const int rv = lda / (16 / esz);
  const int ns = (rv + 31) / 32;            // slabs of 32 row vectors
  *nsw = (ns + rpt - 1) / rpt;              // warps per column group
  *groups = kConsumerWarps / *nsw;          // column groups
}

struct RowsLayout {
  SmemLayout s;    // stages (A tile + per-column vector tiles), barriers, reduction buffer
  int part_off;    // [2][nsw][nb] float2 partial dots
  int v_off;       // v as FP32 (hi) and, for the double-float passes, its low parts: [2][lda]
  int total;
};

__host__ __device__ inline RowsLayout rows_layout(int lda, int esz, int nb, int stages, int nsw) {
  RowsLayout R;
  R.s = make_layout(lda, esz, nb, stages, 0);
  R.part_off = R.s.total;
  R.v_off = R.part_off + align_up_i(2 * nsw * nb * 8, 128);
  R.total = R.v_off + align_up_i(2 * lda * 4, 128);
  return R;
}

// bar.red.or over the consumer warps (named barrier 1): every consumer thread
// gets the OR of `pred`; shared-memory writes before it are visible after it.
__device__ __forceinline__ bool consumers_bar_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)(pred ? 1 : 0)), "n"(kConsumerWarps * 32)
      : "memory");
  return r != 0;
}

// the 16-byte row vector `raw` as VEC FP32 values
template <typename TA>
__device__ __forceinline__ void unpack16(const uint4& raw, float* o);
template <>
__device__ __forceinline__ void unpack16<float>(const uint4& raw, float* o) {
  o[0] = __uint_as_float(raw.x);
  o[1] = __uint_as_float(raw.y);
  o[2] = __uint_as_float(raw.z);
  o[3] = __uint_as_float(raw.w);
}
template <>
__device__ __forceinline__ void unpack16<bf16raw>(const uint4& raw, float* o) {
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[2 * q] = __uint_as_float(w[q] << 16);
    o[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
  }
}

__device__ __forceinline__ dfl cv_pair(const char* stage, const SmemLayout& L, int q, int jj) {
  const float2 v = reinterpret_cast<const float2*>(stage + L.cv_off[q])[jj];
  return {v.x, v.y};
}

}  // namespace

template <typename TA, bool DF, int MODE, int RPT>
__global__ void __launch_bounds__(kFusedThreads, 1) k_rows(const StreamArgs a) {
  constexpr int VEC = VecOf<TA>::N;
  constexpr int CPT = kRowsCPT;
  constexpr int NACC = (MODE == M_RESID) ? 2 : ((MODE == M_ADAT) ? 1 : 0);
  constexpr int NA = NACC > 0 ? NACC : 1;
  using TC = typename std::conditional<DF, double, float>::type;
  extern __shared__ __align__(128) char smem[];
  int nsw, groups;
  rows_geom(a.lda, (int)sizeof(TA), RPT, &nsw, &groups);
  const RowsLayout R = rows_layout(a.lda, (int)sizeof(TA), a.nb, a.stages, nsw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + R.s.bar_off);
  uint64_t* empty = full + a.stages;
  double* red = reinterpret_cast<double*>(smem + R.s.red_off);
  float2* part_s = reinterpret_cast<float2*>(smem + R.part_off);  // [2][nsw][nb]
  __shared__ int s_flag;
  pdl_wait();
  pdl_trigger();
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RV = a.lda / VEC;
  const int S = a.stages;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int grp = warp / nsw, qs = warp % nsw;
  const bool active = warp < kConsumerWarps && grp < groups;
  dfl smu = {0.0f, 0.0f};  // sigma mu as a pair
  if (DF && (MODE == M_RESID || MODE == M_DIR)) {
    const double v = a.sigma * a.sc->mu;
    smu.h = (float)v;
    smu.l = (float)(v - (double)smu.h);
  }
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  // v in shared memory (read once per tile per lane): v_hi[lda], v_lo[lda]
  float* v_hi = reinterpret_cast<float*>(smem + R.v_off);
  float* v_lo = v_hi + a.lda;
  for (int i = tid; i < a.lda; i += blockDim.x) {
    const double v = i < a.m ? a.vin[i] : 0.0;
    v_hi[i] = (float)v;
    v_lo[i] = (float)(v - (double)v_hi[i]);
  }
  __syncthreads();
  // this lane's rows: row vector (qs * RPT + k) * 32 + lane, k < RPT
  float ah[NA][RPT][VEC], al[DF ? NA : 1][DF ? RPT : 1][VEC];
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int e = 0; e < VEC; ++e)
#pragma unroll
      for (int t = 0; t < NA; ++t) {
        ah[t][k][e] = 0.0f;
        if (DF) al[DF ? t : 0][DF ? k : 0][e] = 0.0f;
      }
  bool aborted = false;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int issued = 0, st = 0;
      uint32_t parity = 1u;  // phase of empty[st] to wait for (the first pass waits for none)
      for (int i = 0; i < my_tiles; ++i) {
        if (i >= S && !mbar_wait(&empty[st], parity, a.err)) {
          aborted = true;
          break;
        }
        fence_proxy_async_smem();
        issue_tile<TA>(a, R.s, smem, full, st, (int)blockIdx.x + i * (int)gridDim.x);
        issued = i + 1;
        if (++st == S) {
          st = 0;
          parity ^= 1u;
        }
      }
      if (aborted || *a.err != ERR_NONE)
        for (int j = (issued > S ? issued - S : 0); j < issued; ++j)
          mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), a.err);
    }
  } else {
    // ---------------- consumers ----------------
    // phase 1 of a tile: wait for its stage, form this warp's slab partials
    // of a_j^T v for the group's four columns and write them to partial
    // buffer pb; returns whether the stage's wait succeeded
    auto phase1 = [&](int st, uint32_t parity, int ncols, int pb) -> bool {
      const bool ok = mbar_wait(&full[st], parity, a.err);
      const TA* At = reinterpret_cast<const TA*>(smem + (size_t)st * R.s.stage_bytes);
      // partial dots of the four columns: two interleaved sums per column
      float ph[CPT][2], pl[CPT][2];
#pragma unroll
      for (int c = 0; c < CPT; ++c) ph[c][0] = ph[c][1] = pl[c][0] = pl[c][1] = 0.0f;
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int rv = (qs * RPT + k) * 32 + lane;
        const bool row_ok = ok && active && rv < RV;
        float vk[VEC], vkl[DF ? VEC : 1];
#pragma unroll
        for (int e = 0; e < VEC; e += 4) {
          const float4 t4 = row_ok ? *reinterpret_cast<const float4*>(v_hi + rv * VEC + e)
                                   : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          vk[e] = t4.x;
          vk[e + 1] = t4.y;
          vk[e + 2] = t4.z;
          vk[e + 3] = t4.w;
          if (DF) {
            const float4 l4 = row_ok ? *reinterpret_cast<const float4*>(v_lo + rv * VEC + e)
                                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            vkl[DF ? e : 0] = l4.x;
            vkl[DF ? e + 1 : 0] = l4.y;
            vkl[DF ? e + 2 : 0] = l4.z;
            vkl[DF ? e + 3 : 0] = l4.w;
          }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int jj = grp * CPT + c;
          uint4 raw = make_uint4(0u, 0u, 0u, 0u);
          if (row_ok && jj < ncols)
            raw = *reinterpret_cast<const uint4*>(At + (size_t)jj * a.lda + (size_t)rv * VEC);
          float av[VEC];
          unpack16<TA>(raw, av);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            if (DF) df_fma(av[e], vk[e], vkl[DF ? e : 0], ph[c][e & 1], pl[c][e & 1]);
            else ph[c][e & 1] = fmaf(av[e], vk[e], ph[c][e & 1]);
          }
        }
      }
      float dh[CPT], dl[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        if (DF) {
          df_add(ph[c][0], pl[c][0], ph[c][1], pl[c][1]);
          dh[c] = ph[c][0];
          dl[c] = pl[c][0];
        } else {
          dh[c] = ph[c][0] + ph[c][1];
          dl[c] = 0.0f;
        }
      }
      // reduce-scatter of the four column sums over the warp: after the steps
      // over lane bits 4 and 3, lane l holds column 2 (l >> 4) + ((l >> 3) & 1)
      // summed over a lane pair / quad, then bits 2..0 complete the sum
      const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
      float xh[2], xl[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float sh = b4 ? dh[q] : dh[q + 2], sl = b4 ? dl[q] : dl[q + 2];
        xh[q] = b4 ? dh[q + 2] : dh[q];
        xl[q] = b4 ? dl[q + 2] : dl[q];
        const float oh = __shfl_xor_sync(0xffffffffu, sh, 16);
        if (DF) df_add(xh[q], xl[q], oh, __shfl_xor_sync(0xffffffffu, sl, 16));
        else xh[q] += oh;
      }
      float yh = b3 ? xh[1] : xh[0], yl = b3 ? xl[1] : xl[0];
      {
        const float sh = b3 ? xh[0] : xh[1], sl = b3 ? xl[0] : xl[1];
        const float oh = __shfl_xor_sync(0xffffffffu, sh, 8);
        if (DF) df_add(yh, yl, oh, __shfl_xor_sync(0xffffffffu, sl, 8));
        else yh += oh;
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, yh, o);
        if (DF) df_add(yh, yl, oh, __shfl_xor_sync(0xffffffffu, yl, o));
        else yh += oh;
      }
      const int c = 2 * (lane >> 4) + ((lane >> 3) & 1);
      const int jj = grp * CPT + c;
      if (ok && active && (lane & 7) == 0 && jj < ncols)
        part_s[(size_t)pb * nsw * a.nb + (size_t)qs * a.nb + jj] = make_float2(yh, DF ? yl : 0.0f);
      return ok;
    };
    // the rest of the tile once its partials are published: the column scalars
    // (lanes 8c .. 8c+7 sum column c's nsw slab partials by a fixed tree, lane
    // 8c forms t_c), then acc += a_j t_j from `raw`, then release the stage
    auto finish = [&](int st, long long j0, int ncols, int pb) {
      const char* stage = smem + (size_t)st * R.s.stage_bytes;
      const float2* pbuf = part_s + (size_t)pb * nsw * a.nb;
      const int c = lane >> 3, q0 = lane & 7;
      const int jj = grp * CPT + c;
      const bool col_ok = active && jj < ncols;
      float sh = 0.0f, sl = 0.0f;
      if (col_ok)
        for (int q = q0; q < nsw; q += 8) {
          const float2 p = pbuf[(size_t)q * a.nb + jj];
          if (DF) df_add(sh, sl, p.x, p.y);
          else sh += p.x;
        }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
        if (DF) df_add(sh, sl, oh, __shfl_xor_sync(0xffffffffu, sl, o));
        else sh += oh;
      }
      float t0h = 0.0f, t0l = 0.0f, t1h = 0.0f, t1l = 0.0f;
      if (col_ok && q0 == 0) {
        const long long j = j0 + jj;
        if (!DF) {
          t0h = reinterpret_cast<const float*>(stage + R.s.cv_off[0])[jj] * sh;
        } else {
          const dfl dot = dfl_make(sh, sl);
          dfl t0 = {0.0f, 0.0f}, t1 = {0.0f, 0.0f};
          if (MODE == M_ADAT) {
            t0 = dfl_mul(cv_pair(stage, R.s, 0, jj), dot);
          } else if (MODE == M_RESID) {
            const dfl x = cv_pair(stage, R.s, 0, jj);
            const dfl s = cv_pair(stage, R.s, 1, jj);
            const dfl cc = cv_pair(stage, R.s, 2, jj);
            const dfl rd = dfl_sub(dfl_add(dot, s), cc);
            const dfl d2 = dfl_div(x, s);
            if (qs == 0) {
              a.out_df[0][j] = make_float2(rd.h, rd.l);
              a.out_df[1][j] = make_float2(d2.h, d2.l);
            }
            t0 = x;
            const dfl xc = dfl_sub(x, dfl_div(smu, s));
            t1 = a.feasible ? xc : dfl_sub(xc, dfl_mul(d2, rd));
          } else if (MODE == M_DIR) {
            const dfl x = cv_pair(stage, R.s, 0, jj);
            const dfl s = cv_pair(stage, R.s, 1, jj);
            const dfl v = cv_pair(stage, R.s, 2, jj);
            const dfl rd = a.feasible ? dfl{0.0f, 0.0f} : cv_pair(stage, R.s, 3, jj);
            const dfl ds = dfl_neg(dfl_add(rd, dot));
            // dx = -x + (sigma mu - x ds - v) / s
            const dfl num = dfl_sub(dfl_sub(smu, dfl_mul(x, ds)), v);
            const dfl dx = dfl_sub(dfl_div(num, s), x);
            if (qs == 0) {
              a.out_df[0][j] = make_float2(dx.h, dx.l);
              a.out_df[1][j] = make_float2(ds.h, ds.l);
            }
          }
          t0h = t0.h;
          t0l = t0.l;
          t1h = t1.h;
          t1l = t1.l;
        }
      }
      if (NACC > 0) {
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const float th = __shfl_sync(0xffffffffu, t0h, cc * 8);
          const float tl = DF ? __shfl_sync(0xffffffffu, t0l, cc * 8) : 0.0f;
          float uh = 0.0f, ul = 0.0f;
          if (NACC > 1) {
            uh = __shfl_sync(0xffffffffu, t1h, cc * 8);
            ul = __shfl_sync(0xffffffffu, t1l, cc * 8);
          }
          const int jj2 = grp * CPT + cc;
#pragma unroll
          for (int k = 0; k < RPT; ++k) {
            // the column slice again from the stage (still held: this warp
            // has not released it), rather than kept in registers
            const int rv = (qs * RPT + k) * 32 + lane;
            uint4 raw = make_uint4(0u, 0u, 0u, 0u);
            if (active && rv < RV && jj2 < ncols)
              raw = *reinterpret_cast<const uint4*>(reinterpret_cast<const TA*>(stage) + (size_t)jj2 * a.lda +
                                                    (size_t)rv * VEC);
            float av[VEC];
            unpack16<TA>(raw, av);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
              if (DF) {
                df_fma(av[e], th, tl, ah[0][k][e], al[0][DF ? k : 0][e]);
                if (NACC > 1) df_fma(av[e], uh, ul, ah[NA - 1][k][e], al[DF ? NA - 1 : 0][DF ? k : 0][e]);
              } else {
                ah[0][k][e] = fmaf(av[e], th, ah[0][k][e]);
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    };
    // phase 1, publish, finish, one tile at a time; the stage index, its
    // parity and the tile's first column advance incrementally
    int st = 0, pb = 0;
    uint32_t parity = 0;
    long long j0 = (long long)blockIdx.x * a.nb;
    const long long jstep = (long long)gridDim.x * a.nb;
    for (int i = 0; i < my_tiles; ++i) {
      const int ncols = (int)min((long long)a.nb, a.n - j0);
      const bool ok = phase1(st, parity, ncols, pb);
      if (consumers_bar_or(!ok)) {
        aborted = true;
        break;
      }
      finish(st, j0, ncols, pb);
      j0 += jstep;
      pb ^= 1;
      if (++st == S) {
        st = 0;
        parity ^= 1u;
      }
    }
  }
  aborted = __syncthreads_or(aborted) != 0;

  // ---- per-CTA partials: the column groups' sums of the same rows, in group order ----
#pragma unroll
  for (int t = 0; t < NACC; ++t) {
    float2* buf2 = reinterpret_cast<float2*>(smem);
    float* buf1 = reinterpret_cast<float*>(smem);
    if (active) {
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int rv = (qs * RPT + k) * 32 + lane;
        if (rv < RV)
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const size_t idx = (size_t)grp * a.lda + rv * VEC + e;
            if (DF) buf2[idx] = make_float2(ah[t][k][e], al[DF ? t : 0][DF ? k : 0][e]);
            else buf1[idx] = ah[t][k][e];
          }
      }
    }
    __syncthreads();
    TC* part = static_cast<TC*>(a.partials) + (size_t)blockIdx.x * 2 * a.lda + (size_t)t * a.lda;
    for (int r = tid; r < a.lda; r += blockDim.x) {
      if (DF) {
        float h = buf2[r].x, l = buf2[r].y;
        for (int g = 1; g < groups; ++g) df_add(h, l, buf2[(size_t)g * a.lda + r].x, buf2[(size_t)g * a.lda + r].y);
        part[r] = aborted ? (TC)0 : (TC)((double)h + (double)l);
      } else {
        float s = buf1[r];
        for (int g = 1; g < groups; ++g) s += buf1[(size_t)g * a.lda + r];
        part[r] = aborted ? (TC)0 : (TC)s;
      }
    }
    __syncthreads();
  }
  if (a.epilogue == E_NONE) return;
  if (tree_reduce<TC>(a, NACC, &s_flag)) stream_epilogue<TC>(a, NACC, red);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
RowsPlan make_rows_plan(int lda, long long n, int esz, int num_sms, bool df) {
  RowsPlan p;
  if (esz != 4 && esz != 2) return p;
  const int rv = lda / (16 / esz);
  const int ns = (rv + 31) / 32;
  // slabs per warp: as few as cover the rows with 16 warps; the FP32 product
  // takes two when it can, so that each lane's share of a column (and of the
  // per-column overhead: addressing, reductions) doubles, while the
  // double-float passes need the registers for their accumulator pairs
  p.rpt = (ns + kConsumerWarps - 1) / kConsumerWarps;
  if (!df && ns >= 2) p.rpt = std::max(p.rpt, 2);
  if (p.rpt < 1 || p.rpt > 2) return p;
  int nsw = 0, groups = 0;
  rows_geom(lda, esz, p.rpt, &nsw, &groups);
  if (groups < 1) return p;
  p.nb = kRowsCPT * groups;
  p.ntiles = (int)((n + p.nb - 1) / p.nb);
  const int budget = 220 * 1024;
  int stages = kRowsMaxStages;
  for (; stages >= 2; --stages) {
    const RowsLayout R = rows_layout(lda, esz, p.nb, stages, nsw);
    // the end-of-kernel combine buffer ([groups][lda] pairs) reuses the stage area
    if (R.total <= budget && (long long)stages * R.s.stage_bytes >= (long long)groups * lda * 8) break;
  }
  if (stages < 2) return p;
  p.stages = stages;
  p.smem = rows_layout(lda, esz, p.nb, stages, nsw).total;
  p.grid = std::max(1, std::min(std::min(p.ntiles, num_sms), kGroup * kMaxGroups));
  p.ok = p.smem <= 227 * 1024 && p.ntiles >= 1;
  return p;
}

namespace {
template <typename TA, bool DF, int MODE, int RPT>
cudaError_t rows_launch_t(StreamArgs a, const RowsPlan& p, cudaStream_t st, bool pdl) {
  a.nb = p.nb;
  a.ntiles = p.ntiles;
  a.stages = p.stages;
  auto k = k_rows<TA, DF, MODE, RPT>;
  cudaError_t e = ensure_smem((const void*)k, p.smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  e = launch_maybe_pdl(k, dim3(p.grid), dim3(kFusedThreads), (size_t)p.smem, st, pdl, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename TA, bool DF, int MODE>
cudaError_t rows_rpt(const StreamArgs& a, const RowsPlan& p, cudaStream_t st, bool pdl) {
  if (p.rpt == 1) return rows_launch_t<TA, DF, MODE, 1>(a, p, st, pdl);
  if (p.rpt == 2) return rows_launch_t<TA, DF, MODE, 2>(a, p, st, pdl);
  return cudaErrorInvalidValue;
}

template <typename TA>
cudaError_t rows_mode(bool df, int mode, const StreamArgs& a, const RowsPlan& p, cudaStream_t st,
                      bool pdl) {
  if (!df) return mode == M_ADAT ? rows_rpt<TA, false, M_ADAT>(a, p, st, pdl) : cudaErrorInvalidValue;
  switch (mode) {
    case M_ADAT: return rows_rpt<TA, true, M_ADAT>(a, p, st, pdl);
    case M_RESID: return rows_rpt<TA, true, M_RESID>(a, p, st, pdl);
    case M_DIR: return rows_rpt<TA, true, M_DIR>(a, p, st, pdl);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_rows(int dtype, bool df, int mode, const StreamArgs& a, const RowsPlan& p,
                        cudaStream_t st, bool pdl) {
  if (!p.ok) return cudaErrorInvalidValue;
  if (dtype == 1) return rows_mode<float>(df, mode, a, p, st, pdl);
  if (dtype == 2) return rows_mode<bf16raw>(df, mode, a, p, st, pdl);
  return cudaErrorInvalidValue;
}

}  // namespace lpk
