// Column-streaming kernels over a dense column-major A (internal header).
//
// Every A-pass of an outer iteration streams column tiles of A (NB columns,
// contiguous because A is column-major with a 16-byte padded leading
// dimension) from HBM into a ring of shared-memory stages with 1-D bulk async
// copies (cp.async.bulk + mbarrier), together with the tiles of the per-column
// vectors the pass needs (d^2, x, s, ...).  One elected thread refills a stage
// as soon as all warps are done with it, so S-1 tiles are always in flight.
//
// Two kernel shapes:
//   * k_adat_fused  -- the hot product u = A diag(d2) A^T v in FP32
//     arithmetic (Section 3's matrix-vector products, eq. normal): each warp
//     takes whole columns: lanes load the column from shared memory into
//     registers once, form d2_j (a_j^T v) with a warp reduction, and
//     accumulate a_j * t_j into per-lane registers that cover all m rows.
//     Shared memory is read once per element.
//   * k_stream      -- the FP64 passes (residuals and right-hand side,
//     directions, FP64 products for the residual refresh): phase 1 forms the
//     per-column dots warp-per-column, phase 2 lets each thread own a slice of
//     rows and accumulate over the tile's columns.  FP64 arithmetic bounds these.
// Both end with a per-CTA partial vector and a "last CTA" reduction in FP64 in
// a fixed order (deterministic), followed by a mode-specific epilogue.
#pragma once

#include "common.cuh"

namespace lpk {

enum StreamMode : int {
  M_ADAT = 0,   // dot with vin; t0 = d2_j * dot; acc0 += a_j t0
  M_AX = 1,     // t0 = cv0_j; acc0 += a_j t0 (no dot)
  M_RESID = 2,  // dot y; rd_j = dot + s_j - c_j; t0 = x_j; t1 = x_j - sm/s_j - d2_j rd_j
  M_DIR = 3,    // dot dy; ds_j = -rd_j - dot; dx_j = -x_j + sm/s_j - d2_j ds_j - v_j/s_j
  M_ATY = 4,    // out0_j = dot(a_j, vin)
};

enum Epilogue : int {
  E_NONE = 0,
  E_PLAIN = 1,      // out_m0 = sum acc0 (and out_m1 = sum acc1)
  E_PCG_A = 2,      // q = sum acc0; pq = p.q; alpha = rho/pq; dy += alpha p; r -= alpha q
  E_TRUE_RES = 3,   // r = rhs - sum acc0  (true residual of the normal equations)
  E_RESID = 4,      // rp = acc0 - b; p = acc1 - rp (infeasible) or acc1 (feasible); scalars
  E_DIR = 5,        // c1, c2 from the column reductions
  E_CHEB = 6,       // Chebyshev residual update r -= sum acc0
};

struct StreamArgs {
  const void* A;
  int lda;           // padded leading dimension (elements), multiple of 16 bytes
  int m;
  long long n;
  int nb;            // columns per tile
  int ntiles;
  int stages;
  int feasible;
  double sigma;      // centering parameter; mu is read from sc->mu
  const void* cv[kMaxColVecs];  // per-column inputs, padded device vectors
  int cv_esz[kMaxColVecs];      // 4 or 8 bytes
  int ncv;
  const double* vin;  // m-vector for the column dots
  double* out_col[2];  // per-column FP64 outputs (n)
  float2* out_df[2];   // per-column double-float outputs (n) of the double-float kernels
  int pdl;             // host side: launch with programmatic stream serialization
  float* out_colf;     // per-column FP32 output (n)
  void* partials;      // [grid][lda] of TC per accumulator (acc1 after acc0)
  double* red_partials;  // [grid][2] column reductions
  unsigned* ticket;
  int epilogue;
  // epilogue operands (m-vectors unless stated)
  double* out_m0;
  double* out_m1;
  const double* bvec;  // b (E_RESID) or the normal-equation rhs (E_TRUE_RES)
  double* pcg_p;
  double* pcg_r;
  double* pcg_dy;
  DevScalars* sc;
  int* err;
  int skip_level;      // return at once if sc->inner_done >= skip_level (0: never)
  double* coef;        // E_PCG_A: alpha of CG step j stored at coef[2j] (Lanczos interval)
  const long long* colptr;  // CSC: n+1 column pointers
  const int* rowidx;        // CSC: row indices
  const void* spval;        // CSC: values (FP32 or FP64)
  // sparse A by rows as well (the deterministic two-pass product): CSR arrays,
  // row segments of at most kSegNnz entries, per-column scalars and segment sums
  const long long* rowptr;  // m+1
  const int* colidx;        // CSR column indices
  const void* rval;         // CSR values
  const long long* seg;     // [nseg][2]: first and last+1 CSR index of a segment
  const int* seg_row;       // row of a segment
  const int* row_seg;       // m+1: the segments of row i are row_seg[i] .. row_seg[i+1]-1
  int nseg;
  void* tcol;               // [2][n] per-column scalars t0, t1 (TC)
  double* segsum;           // [nseg][2] segment sums
  double* gpart;       // [ceil(grid/kGroup)][2][lda] group sums of the partials (FP64, or FP32
                       // pairs in the same 8 bytes when the partials are FP32)
  unsigned* gtickets;  // [kMaxGroups + 1] self-resetting tickets of the two-level reduction
};

// Shared-memory layout shared by host and device.
struct SmemLayout {
  int stage_bytes;   // A tile + per-column vector tiles
  int a_bytes;       // A tile bytes for a full tile
  int cv_off[kMaxColVecs];
  int bar_off;       // S mbarriers
  int v_off;         // vin as TC (lda entries)
  int t_off;         // per-tile column scalars (2 * nb doubles)
  int red_off;       // small reduction buffer (64 doubles)
  int total;
};

__host__ __device__ inline int align_up_i(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout make_layout(int lda, int esz, int nb, int stages,
                                                  int tc_bytes) {
  SmemLayout L;
  L.a_bytes = nb * lda * esz;
  int off = align_up_i(L.a_bytes, 128);
  for (int q = 0; q < kMaxColVecs; ++q) {
    L.cv_off[q] = off;
    off += align_up_i(nb * 8, 128);
  }
  L.stage_bytes = off;
  off = stages * L.stage_bytes;
  L.bar_off = off;
  off += align_up_i(2 * stages * 8, 128);  // full[] and empty[] barriers
  L.v_off = off;
  off += align_up_i(lda * tc_bytes, 128);
  L.t_off = off;
  off += align_up_i(2 * nb * 8, 128);
  L.red_off = off;
  off += 64 * 8;
  L.total = off;
  return L;
}

}  // namespace lpk
