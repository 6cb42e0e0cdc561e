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
//   * each of the m/32 pivot steps is three launches: one CTA of 32 x 32
//     threads sweeps the 32 x 32 pivot block (the step's serial chain of 32
//     pivots, one element per thread), one launch forms the panel
//     U_I = A_{I,K} (-P^{-1}) of every row block once, and one launch over the
//     upper-triangle 32 x 32 tiles writes the next iterate (each tile and its
//     mirror: the iterate is symmetric; 128 threads per tile, a 2 x 4 block of
//     outputs each); two buffers alternate, so no tile is read after it is
//     overwritten.
#include "internal.h"
#include "df.cuh"

namespace lpk {

namespace {
constexpr int SB = 32;          // pivot block = tile
constexpr int SW_THREADS = 256; // threads of the panel kernel: 4 outputs each
// The tile kernel: ST_THREADS threads per 32 x 32 tile (2 x 4 outputs each),
// kStepTiles tiles per CTA, each with its own shared memory and named barrier;
// a CTA covers several tiles, so the kernel leaves SMs free for the pivot
// kernel running beside it.
constexpr int ST_THREADS = 128;
constexpr int kStepTiles = 4;

// the operands and the transposed tile of one tile of k_sweep_step, as (hi, lo) pairs
struct StepSmem {
  float2 P[SB][SB + 1];  // -P^{-1} or U_I
  float2 C[SB][SB + 1];  // A_{J,K}
  float2 T[SB][SB + 1];  // the tile, for the mirror
};

// barrier over the `count` threads of one part of the CTA (ids >= 1; 0 is
// __syncthreads')
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

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

// The pivot block of step K swept on its 32 pivots: -P_K^{-1} into (qh, ql)
// and the pivots (the squares of the Cholesky diagonal) into piv.  For K = 0,
// P_0 is tile (0, 0) of the iterate x.  For K >= 1, x is the iterate that step
// K-1 reads, and P_K = A_KK + U A_{K,K-1}^T with U = A_{K,K-1} (-P_{K-1}^{-1})
// ((qph, qpl)): the operations, in the order, by which k_sweep_step forms tile
// (K, K) of the next iterate, so both hold the same values and this kernel can
// run beside step K-1's tile kernel.  One CTA of SB x SB threads, thread (a, b)
// owning entry (a, b); per pivot t every thread reads d = P_tt, P_at and P_bt
// from one copy of the block and writes its new entry to the other (a == t or
// b == t: the scaled column or -1/d; otherwise P_ab - (P_at/d) P_bt).
__global__ void __launch_bounds__(SB* SB) k_sweep_pivot(const float* __restrict__ xh, const float* __restrict__ xl,
                                                       int mp, int K, const float* __restrict__ qph,
                                                       const float* __restrict__ qpl, float* __restrict__ qh,
                                                       float* __restrict__ ql, float* __restrict__ piv) {
  __shared__ float Ph[SB][SB + 1], Pl[SB][SB + 1];
  __shared__ float Th[SB][SB + 1], Tl[SB][SB + 1];  // A_{K,K-1}, then U
  __shared__ float Ch[SB][SB + 1], Cl[SB][SB + 1];  // A_{K,K-1}
  __shared__ float Qh[SB][SB + 1], Ql[SB][SB + 1];  // -P_{K-1}^{-1}
  const int a = threadIdx.x / SB, b = threadIdx.x % SB;
  const int k0 = K * SB;
  const size_t akk = (size_t)(k0 + a) * mp + k0 + b;
  if (K == 0 || !qph) {
    Ph[a][b] = xh[akk];
    Pl[a][b] = xl[akk];
    __syncthreads();
  } else {
    const size_t akp = (size_t)(k0 + a) * mp + (k0 - SB) + b;
    Th[a][b] = xh[akp];
    Tl[a][b] = xl[akp];
    Ch[a][b] = xh[akp];
    Cl[a][b] = xl[akp];
    Qh[a][b] = qph[a * SB + b];
    Ql[a][b] = qpl[a * SB + b];
    float oh = xh[akk], ol = xl[akk];
    __syncthreads();
    float uh = 0.0f, ul = 0.0f;
    for (int c = 0; c < SB; ++c) df_mac(Th[a][c], Tl[a][c], Qh[c][b], Ql[c][b], uh, ul);
    df_renorm(uh, ul);
    __syncthreads();  // every read of T is done
    Th[a][b] = uh;
    Tl[a][b] = ul;
    __syncthreads();
    for (int c = 0; c < SB; ++c) df_mac(Th[a][c], Tl[a][c], Ch[b][c], Cl[b][c], oh, ol);
    df_renorm(oh, ol);
    Ph[a][b] = oh;
    Pl[a][b] = ol;
    __syncthreads();
  }
  // the 32 pivots, reading one copy of the block and writing the other (the
  // Q buffers are free by now), so one barrier per pivot suffices
  float(*ch)[SB + 1] = Ph;
  float(*cl)[SB + 1] = Pl;
  float(*nh)[SB + 1] = Qh;
  float(*nl)[SB + 1] = Ql;
  for (int t = 0; t < SB; ++t) {
    const float dh = ch[t][t], dl = cl[t][t];
    const float ah = ch[a][t], al = cl[a][t];
    const float bh = ch[b][t], bl = cl[b][t];
    float h = ch[a][b], l = cl[a][b];
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
    nh[a][b] = h;
    nl[a][b] = l;
    __syncthreads();
    float(*th)[SB + 1] = ch;
    float(*tl)[SB + 1] = cl;
    ch = nh;
    cl = nl;
    nh = th;
    nl = tl;
  }
  qh[a * SB + b] = ch[a][b];
  ql[a * SB + b] = cl[a][b];
}

// The panel of pivot step K: U_I = A_{I,K} (-P_K^{-1}) for every row block I
// != K (one 32 x 32 block per CTA, 4 outputs per thread), from the iterate
// step K reads and the swept pivot block.  Every tile of step K in row block I
// uses U_I, so it is formed once here instead of once per tile.
__global__ void __launch_bounds__(SW_THREADS) k_sweep_panel(const float* __restrict__ sh_, const float* __restrict__ sl_,
                                                            int mp, int K, const float* __restrict__ qh,
                                                            const float* __restrict__ ql, float* __restrict__ uh_,
                                                            float* __restrict__ ul_, float* __restrict__ uth_,
                                                            float* __restrict__ utl_) {
  __shared__ float Ph[SB][SB + 1], Pl[SB][SB + 1];
  __shared__ float Th[SB][SB + 1], Tl[SB][SB + 1];
  const int I = blockIdx.x;
  if (I == K) return;
  const int tid = threadIdx.x, k0 = K * SB;
  for (int e = tid; e < SB * SB; e += SW_THREADS) {
    const int a = e / SB, b = e % SB;
    Ph[a][b] = qh[e];
    Pl[a][b] = ql[e];
    const size_t src = (size_t)(I * SB + a) * mp + k0 + b;
    Th[a][b] = sh_[src];
    Tl[a][b] = sl_[src];
  }
  __syncthreads();
  const int r = tid >> 3, c4 = (tid & 7) * 4;
  float uh4[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ul4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int b = 0; b < SB; ++b) {
    const float th = Th[r][b], tl = Tl[r][b];
#pragma unroll
    for (int q = 0; q < 4; ++q) df_mac(th, tl, Ph[b][c4 + q], Pl[b][c4 + q], uh4[q], ul4[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    df_renorm(uh4[q], ul4[q]);
    uh_[(size_t)I * SB * SB + r * SB + c4 + q] = uh4[q];
    ul_[(size_t)I * SB * SB + r * SB + c4 + q] = ul4[q];
    if (uth_) {  // U_I^T as well, for the 64 x 64 block kernel's coalesced staging
      uth_[(size_t)I * SB * SB + (c4 + q) * SB + r] = uh4[q];
      utl_[(size_t)I * SB * SB + (c4 + q) * SB + r] = ul4[q];
    }
  }
}

// (I, J) with J >= I of upper-triangle tile number t (column by column)
__device__ __forceinline__ void upper_tile(int t, int* I, int* J) {
  int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((j + 1) * (j + 2) / 2 <= t) ++j;
  while (j * (j + 1) / 2 > t) --j;
  *J = j;
  *I = t - j * (j + 1) / 2;
}

// One pivot step K: src -> dst.  The iterate stays symmetric, so only the
// tiles (I, J) with J >= I are formed (the swept pivot block -P^{-1} from
// k_sweep_pivot, the panels U from k_sweep_panel):
//   I = J = K:      -P^{-1}
//   J = K:          A_IK P^{-1} = -U_I
//   I = K:          P^{-1} A_KJ = -U_J^T
//   otherwise:      A_IJ + U_I A_{J,K}^T
// and each is written to (I, J) and, transposed through shared memory, to
// (J, I); both writes are coalesced 16-byte stores along rows.  A tile takes
// ST_THREADS threads, each forming a 2 x 4 block of outputs from operands held
// in shared memory as (hi, lo) pairs, so one 8-byte load brings both halves
// and every operand loaded serves four or two multiply-adds; kStepTiles tiles
// share a CTA, each with its own named barrier.  Every output is formed by the
// same operations in the same order as before this blocking (and as the pivot
// kernel forms the next pivot block), so the results are unchanged.
__global__ void __launch_bounds__(ST_THREADS* kStepTiles) k_sweep_step(const float* __restrict__ sh_, const float* __restrict__ sl_,
                                                                       float* __restrict__ dh_, float* __restrict__ dl_,
                                                                       int mp, int K, const float* __restrict__ qh,
                                                                       const float* __restrict__ ql,
                                                                       const float* __restrict__ uh_,
                                                                       const float* __restrict__ ul_,
                                                                       int tiles_per_cta) {
  extern __shared__ __align__(16) char sw_smem[];
  const int part = threadIdx.x / ST_THREADS;
  StepSmem& S = reinterpret_cast<StepSmem*>(sw_smem)[part];
  const int nt = mp / SB;
  const int tile = blockIdx.x * tiles_per_cta + part;
  if (tile >= nt * (nt + 1) / 2) return;  // no tile for this part; the others' barriers count their own threads
  int I, J;
  upper_tile(tile, &I, &J);
  const int k0 = K * SB;
  const int tid = threadIdx.x % ST_THREADS;
  const int bar = 1 + part;
  const int r2 = (tid >> 3) * 2, c4 = (tid & 7) * 4;  // outputs: rows r2, r2 + 1; columns c4 .. c4 + 3

  // ---- operands: P <- -P^{-1} or U_I, C <- A_{J,K} ----
  for (int e = tid; e < SB * SB; e += ST_THREADS) {
    const int a = e / SB, b = e % SB;
    if (I == K && J == K) {
      S.P[a][b] = make_float2(qh[e], ql[e]);
    } else if (J == K) {
      S.P[a][b] = make_float2(uh_[(size_t)I * SB * SB + e], ul_[(size_t)I * SB * SB + e]);
    } else if (I == K) {
      S.P[a][b] = make_float2(uh_[(size_t)J * SB * SB + e], ul_[(size_t)J * SB * SB + e]);
    } else {
      S.P[a][b] = make_float2(uh_[(size_t)I * SB * SB + e], ul_[(size_t)I * SB * SB + e]);
      const size_t src = (size_t)(J * SB + a) * mp + k0 + b;
      S.C[a][b] = make_float2(sh_[src], sl_[src]);
    }
  }
  named_sync(bar, ST_THREADS);

  // ---- this thread's 2 x 4 outputs ----
  float oh[2][4], ol[2][4];
  if (I == K && J == K) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 v = S.P[r2 + a][c4 + q];
        oh[a][q] = v.x;
        ol[a][q] = v.y;
      }
  } else if (J == K) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 v = S.P[r2 + a][c4 + q];
        oh[a][q] = -v.x;
        ol[a][q] = -v.y;
      }
  } else if (I == K) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 v = S.P[c4 + q][r2 + a];
        oh[a][q] = -v.x;
        ol[a][q] = -v.y;
      }
  } else {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const size_t src = (size_t)(I * SB + r2 + a) * mp + J * SB + c4;
      const float4 h4 = *reinterpret_cast<const float4*>(sh_ + src);
      const float4 l4 = *reinterpret_cast<const float4*>(sl_ + src);
      oh[a][0] = h4.x; oh[a][1] = h4.y; oh[a][2] = h4.z; oh[a][3] = h4.w;
      ol[a][0] = l4.x; ol[a][1] = l4.y; ol[a][2] = l4.z; ol[a][3] = l4.w;
    }
    for (int b = 0; b < SB; ++b) {
      const float2 t0 = S.P[r2][b], t1 = S.P[r2 + 1][b];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 cv = S.C[c4 + q][b];
        df_mac(t0.x, t0.y, cv.x, cv.y, oh[0][q], ol[0][q]);
        df_mac(t1.x, t1.y, cv.x, cv.y, oh[1][q], ol[1][q]);
      }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) df_renorm(oh[a][q], ol[a][q]);
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const size_t dst = (size_t)(I * SB + r2 + a) * mp + J * SB + c4;
    *reinterpret_cast<float4*>(dh_ + dst) = make_float4(oh[a][0], oh[a][1], oh[a][2], oh[a][3]);
    *reinterpret_cast<float4*>(dl_ + dst) = make_float4(ol[a][0], ol[a][1], ol[a][2], ol[a][3]);
  }
  if (I == J) return;
  // the mirror (J, I) = tile^T, through shared memory
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) S.T[r2 + a][c4 + q] = make_float2(oh[a][q], ol[a][q]);
  named_sync(bar, ST_THREADS);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    float2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = S.T[c4 + q][r2 + a];
    const size_t dst = (size_t)(J * SB + r2 + a) * mp + I * SB + c4;
    *reinterpret_cast<float4*>(dh_ + dst) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
    *reinterpret_cast<float4*>(dl_ + dst) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
  }
}

// The same pivot step for large matrices, on 64 x 64 blocks of the upper
// triangle (2 x 2 tiles of 32) with 256 threads, each forming a 4 x 4 block
// of outputs.  The operands of an interior tile, U of the block's two row
// tiles and A_{J,K} of its two column tiles, are held transposed in shared
// memory ([k][row] pairs), so a thread's four rows and four columns come in
// two 16-byte loads each and every loaded pair serves four multiply-adds.
// Every output is formed by the same operations in the same order as in
// k_sweep_step.  Tiles of row or column K are copied from the pivot block or
// the panel; a diagonal block forms its upper-right tile and mirrors it into
// the lower-left one, an off-diagonal block is mirrored whole, through shared
// memory.  One 64 x 64 block per CTA: about one wave of CTAs for the
// 2048-row factor, where the 32 x 32 tiles take two.
namespace {
constexpr int SB2 = 2 * SB;        // 64
constexpr int S64_THREADS = 256;   // 16 x 16 threads, 4 x 4 outputs each
struct Step64Smem {
  union {
    struct {
      float2 U[SB][SB2];   // [k][row]: U of row tiles 2 I2, 2 I2 + 1
      float2 C[SB][SB2];   // [k][col]: A_{J,K} of column tiles 2 J2, 2 J2 + 1
    } op;
    float2 T[SB2][SB2 + 1];  // the block, for the mirror
  };
};
}  // namespace

__global__ void __launch_bounds__(S64_THREADS, 4) k_sweep_step64(const float* __restrict__ sh_, const float* __restrict__ sl_,
                                                                 float* __restrict__ dh_, float* __restrict__ dl_,
                                                                 int mp, int K, const float* __restrict__ qh,
                                                                 const float* __restrict__ ql,
                                                                 const float* __restrict__ uh_,
                                                                 const float* __restrict__ ul_,
                                                                 const float* __restrict__ uth_,
                                                                 const float* __restrict__ utl_) {
  extern __shared__ __align__(16) char s64_smem[];
  Step64Smem& S = *reinterpret_cast<Step64Smem*>(s64_smem);
  const int nt = mp / SB, nb = nt / 2;
  int I2, J2;
  upper_tile(blockIdx.x, &I2, &J2);
  if (I2 >= nb || J2 >= nb) return;
  const int k0 = K * SB;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int r4 = ty * 4, c4 = tx * 4;            // rows / columns within the 64 x 64 block
  const int qa = r4 >> 5, qb = c4 >> 5;          // this thread's quadrant
  const int I = 2 * I2 + qa, J = 2 * J2 + qb;    // its tile
  const int r = r4 & (SB - 1), c = c4 & (SB - 1);  // rows / columns within the tile
  const bool lower_of_diag = I2 == J2 && qa > qb;  // formed as the mirror of the upper-right tile

  // ---- operands of the interior tiles, transposed: U from the panel's
  // transposed copy, A_{J,K}^T as the iterate's row block K (the iterate is
  // stored symmetric: off-diagonal tiles are written with their mirror), so
  // consecutive threads read consecutive addresses and store to consecutive
  // banks ----
  for (int e = tid; e < SB2 * SB; e += S64_THREADS) {
    const int k = e / SB2, row = e % SB2;  // k in [0, 32), row of the block's row (column) pair
    const int ti = 2 * I2 + row / SB, tj = 2 * J2 + row / SB;
    const size_t ue = (size_t)ti * SB * SB + (size_t)k * SB + (row % SB);
    S.op.U[k][row] = ti == K ? make_float2(0.0f, 0.0f) : make_float2(uth_[ue], utl_[ue]);
    const size_t ce = (size_t)(k0 + k) * mp + tj * SB + (row % SB);
    S.op.C[k][row] = make_float2(sh_[ce], sl_[ce]);
  }
  __syncthreads();

  float oh[4][4], ol[4][4];
  if (!lower_of_diag) {
    if (I == K && J == K) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4 h4 = *reinterpret_cast<const float4*>(qh + (r + a) * SB + c);
        const float4 l4 = *reinterpret_cast<const float4*>(ql + (r + a) * SB + c);
        oh[a][0] = h4.x; oh[a][1] = h4.y; oh[a][2] = h4.z; oh[a][3] = h4.w;
        ol[a][0] = l4.x; ol[a][1] = l4.y; ol[a][2] = l4.z; ol[a][3] = l4.w;
      }
    } else if (J == K) {  // -U_I
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const size_t u = (size_t)I * SB * SB + (size_t)(r + a) * SB + c;
        const float4 h4 = *reinterpret_cast<const float4*>(uh_ + u);
        const float4 l4 = *reinterpret_cast<const float4*>(ul_ + u);
        oh[a][0] = -h4.x; oh[a][1] = -h4.y; oh[a][2] = -h4.z; oh[a][3] = -h4.w;
        ol[a][0] = -l4.x; ol[a][1] = -l4.y; ol[a][2] = -l4.z; ol[a][3] = -l4.w;
      }
    } else if (I == K) {  // -U_J^T
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const size_t u = (size_t)J * SB * SB + (size_t)(c + q) * SB + (r + a);
          oh[a][q] = -uh_[u];
          ol[a][q] = -ul_[u];
        }
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const size_t src = (size_t)(I * SB + r + a) * mp + J * SB + c;
        const float4 h4 = *reinterpret_cast<const float4*>(sh_ + src);
        const float4 l4 = *reinterpret_cast<const float4*>(sl_ + src);
        oh[a][0] = h4.x; oh[a][1] = h4.y; oh[a][2] = h4.z; oh[a][3] = h4.w;
        ol[a][0] = l4.x; ol[a][1] = l4.y; ol[a][2] = l4.z; ol[a][3] = l4.w;
      }
      for (int b = 0; b < SB; ++b) {
        const float4 u01 = *reinterpret_cast<const float4*>(&S.op.U[b][r4]);
        const float4 u23 = *reinterpret_cast<const float4*>(&S.op.U[b][r4 + 2]);
        const float4 c01 = *reinterpret_cast<const float4*>(&S.op.C[b][c4]);
        const float4 c23 = *reinterpret_cast<const float4*>(&S.op.C[b][c4 + 2]);
        const float uhv[4] = {u01.x, u01.z, u23.x, u23.z}, ulv[4] = {u01.y, u01.w, u23.y, u23.w};
        const float chv[4] = {c01.x, c01.z, c23.x, c23.z}, clv[4] = {c01.y, c01.w, c23.y, c23.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) df_mac(uhv[a], ulv[a], chv[q], clv[q], oh[a][q], ol[a][q]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) df_renorm(oh[a][q], ol[a][q]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const size_t dst = (size_t)(I * SB + r + a) * mp + J * SB + c;
      *reinterpret_cast<float4*>(dh_ + dst) = make_float4(oh[a][0], oh[a][1], oh[a][2], oh[a][3]);
      *reinterpret_cast<float4*>(dl_ + dst) = make_float4(ol[a][0], ol[a][1], ol[a][2], ol[a][3]);
    }
  }
  // ---- mirrors: the whole block (off-diagonal) or its upper-right tile ----
  __syncthreads();  // every read of the operands is done; T reuses their space
  if (!lower_of_diag) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) S.T[r4 + a][c4 + q] = make_float2(oh[a][q], ol[a][q]);
  }
  __syncthreads();
  // the thread at (r4, c4) of the mirror block writes mirror rows r4.., columns
  // c4.., i.e. the block's entries (c4 + q, r4 + a)
  const bool write_mirror = I2 != J2 || lower_of_diag;
  if (write_mirror) {
    // mirror position: block (J2, I2), its tile rows come from the block's columns
    const int MI = 2 * J2 + qa, MJ = 2 * I2 + qb;  // tile of the mirror entry
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float2 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = S.T[c4 + q][r4 + a];
      const size_t dst = (size_t)(MI * SB + r + a) * mp + MJ * SB + c;
      *reinterpret_cast<float4*>(dh_ + dst) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
      *reinterpret_cast<float4*>(dl_ + dst) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
    }
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
  return 4 * mp * mp + mp + 8 + 4 * SB * SB + 4 * mp * SB;  // + U^T for the block kernel
}

// G: upper triangle of the column-major m x m Gram; qinv: m x m output
cudaError_t launch_sweep_inverse(const double* g, int m, float* scratch, double* qinv, float2* qinv_df,
                                 DevScalars* sc, double rank_tol, int num_sms, cudaStream_t st,
                                 cudaStream_t st_aux, cudaEvent_t ev_x, cudaEvent_t ev_p) {
  const int mp = (m + SB - 1) / SB * SB;
  const size_t mm = (size_t)mp * mp;
  float* a0h = scratch;
  float* a0l = scratch + mm;
  float* a1h = scratch + 2 * mm;
  float* a1l = scratch + 3 * mm;
  float* piv = scratch + 4 * mm;
  // the prescale 2^e, 8-byte aligned after the mp pivots (mp is a multiple of 32)
  double* scale_buf = reinterpret_cast<double*>(scratch + 4 * mm + mp);
  // the swept pivot blocks of steps K (even K: q[0], odd K: q[1]) as pairs
  float* qbase = scratch + 4 * mm + mp + 8;
  float* qh[2] = {qbase, qbase + 2 * SB * SB};
  float* ql[2] = {qbase + SB * SB, qbase + 3 * SB * SB};
  // the panels U_I of the current step: [nt][SB][SB] pairs
  float* uh = qbase + 4 * SB * SB;
  float* ul = uh + (size_t)mp * SB;
  float* uth = ul + (size_t)mp * SB;  // the panels transposed ([nt][k][row] pairs)
  float* utl = uth + (size_t)mp * SB;
  const int g1 = (int)std::max<long long>(1, std::min<long long>(((long long)mm + 255) / 256, (long long)num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_sweep_init<<<g1, 256, 0, st>>>(g, m, mp, a0h, a0l, scale_buf);
  const int nt = mp / SB;
  // tiles per CTA: as many as keep every SM busy (4 when there are tiles for
  // two waves of 4-tile CTAs, fewer for small matrices, down to one per CTA)
  const int ntiles_all = nt * (nt + 1) / 2;
  const int tpc = ntiles_all >= 8 * num_sms ? kStepTiles : (ntiles_all >= 2 * num_sms ? 2 : 1);
  const int tile_smem = (int)(sizeof(StepSmem) * tpc);
  {
    const cudaError_t es = ensure_smem((const void*)k_sweep_step, tile_smem);
    if (es != cudaSuccess) return es;
  }
  // 64 x 64 blocks where the 32 x 32 tiles would take more than one wave of
  // 4-tile CTAs (an even number of tiles per row)
  const bool use64 = (nt % 2) == 0 && ntiles_all >= 8 * num_sms;
  const int nblk64 = (nt / 2) * (nt / 2 + 1) / 2;
  const int smem64 = (int)sizeof(Step64Smem);
  if (use64) {
    const cudaError_t es = ensure_smem((const void*)k_sweep_step64, smem64);
    if (es != cudaSuccess) return es;
  }
  // The pivot kernel of step K + 1 needs the iterate that step K reads and
  // -P_K^{-1}, not step K's output, so with an auxiliary stream it runs beside
  // step K's tile kernel: ev_x marks "the iterate step K reads is complete",
  // ev_p "the pivot kernel of the next step is complete".  Without one, the
  // same kernels run in the same order on st.
  const bool two = st_aux && ev_x && ev_p;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_sweep_pivot<<<1, SB * SB, 0, st>>>(a0h, a0l, mp, 0, nullptr, nullptr, qh[0], ql[0], piv);
  cudaError_t e = cudaSuccess;
  if (two && (e = cudaEventRecord(ev_x, st)) != cudaSuccess) return e;
  for (int K = 0; K < nt; ++K) {
    const bool even = (K & 1) == 0;
    const float* sh = even ? a0h : a1h;
    const float* sl = even ? a0l : a1l;
    if (K + 1 < nt) {
      if (two && (e = cudaStreamWaitEvent(st_aux, ev_x, 0)) != cudaSuccess) return e;
      g_launches.fetch_add(1, std::memory_order_relaxed);
      k_sweep_pivot<<<1, SB * SB, 0, two ? st_aux : st>>>(sh, sl, mp, K + 1, qh[K & 1], ql[K & 1],
                                                          qh[(K + 1) & 1], ql[(K + 1) & 1], piv);
    }
    if (two && K >= 1 && (e = cudaStreamWaitEvent(st, ev_p, 0)) != cudaSuccess) return e;
    g_launches.fetch_add(2, std::memory_order_relaxed);
    k_sweep_panel<<<nt, SW_THREADS, 0, st>>>(sh, sl, mp, K, qh[K & 1], ql[K & 1], uh, ul,
                                             use64 ? uth : nullptr, use64 ? utl : nullptr);
    const int ntiles = nt * (nt + 1) / 2;
    if (use64)
      k_sweep_step64<<<nblk64, S64_THREADS, smem64, st>>>(sh, sl, even ? a1h : a0h, even ? a1l : a0l, mp, K,
                                                          qh[K & 1], ql[K & 1], uh, ul, uth, utl);
    else
      k_sweep_step<<<(ntiles + tpc - 1) / tpc, ST_THREADS * tpc, tile_smem, st>>>(
          sh, sl, even ? a1h : a0h, even ? a1l : a0l, mp, K, qh[K & 1], ql[K & 1], uh, ul, tpc);
    if (two) {
      if ((e = cudaEventRecord(ev_x, st)) != cudaSuccess) return e;
      if (K + 1 < nt && (e = cudaEventRecord(ev_p, st_aux)) != cudaSuccess) return e;
    }
  }
  const bool in0 = (nt & 1) == 0;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const int g2 = (int)std::max<long long>(1, std::min<long long>(((long long)m * m + 255) / 256, (long long)num_sms * 4));
  k_sweep_finish<<<g2, 256, 0, st>>>(in0 ? a0h : a1h, in0 ? a0l : a1l, m, mp, scale_buf, piv, qinv, qinv_df, sc,
                                     rank_tol);
  return cudaGetLastError();
}

}  // namespace lpk
