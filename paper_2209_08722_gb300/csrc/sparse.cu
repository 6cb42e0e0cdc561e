// Column passes over a sparse A in CSC form (col_ptr int64, row_idx int32,
// values FP32 or FP64): the product A diag(d2) A^T v, the residual /
// right-hand-side pass, the direction pass and the CountSketch A D W.
//
// Each CTA owns a contiguous range of columns; a thread takes one column at a
// time (consecutive threads, consecutive columns, so the value / index runs
// of a warp are contiguous in memory).  The m-vector the columns are dotted
// with is gathered from a shared-memory copy; the rank-one updates a_j t_j
// are scattered into per-CTA shared-memory m-vectors with shared-memory
// atomics (4096 FP32 rows = 16 KB), and the per-CTA vectors are reduced by the
// same two-level FP64 tree and epilogues as the dense kernels.  Shared-memory
// atomics make the order of the per-CTA sums depend on scheduling, so sparse
// products agree between runs to rounding, not bitwise.
#include "internal.h"
#include "stream_dev.cuh"

namespace lpk {

template <typename TV, typename TC, int MODE>
__global__ void __launch_bounds__(256) k_sparse(const StreamArgs a) {
  constexpr int NACC = (MODE == M_RESID) ? 2 : ((MODE == M_ADAT || MODE == M_AX) ? 1 : 0);
  constexpr bool DOT = (MODE != M_AX);
  extern __shared__ __align__(16) char smem[];
  TC* v_s = reinterpret_cast<TC*>(smem);
  TC* u0 = v_s + a.lda;
  TC* u1 = u0 + a.lda;
  __shared__ double red[64];
  __shared__ int s_flag;
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const double sigma_mu = a.sigma * a.sc->mu;
  const long long* cp = a.colptr;
  const int* ri = a.rowidx;
  const TV* val = static_cast<const TV*>(a.spval);
  for (int i = tid; i < a.lda; i += blockDim.x) {
    v_s[i] = (DOT && i < a.m) ? (TC)a.vin[i] : (TC)0;
    u0[i] = (TC)0;
    if (NACC > 1) u1[i] = (TC)0;
  }
  __syncthreads();
  const long long per = (a.n + gridDim.x - 1) / gridDim.x;
  const long long j0 = (long long)blockIdx.x * per;
  const long long j1 = min(a.n, j0 + per);
  const double* cv0 = static_cast<const double*>(a.cv[0]);
  const double* cv1 = static_cast<const double*>(a.cv[1]);
  const double* cv2 = static_cast<const double*>(a.cv[2]);
  const double* cv3 = static_cast<const double*>(a.cv[3]);
  double cred0 = 0.0, cred1 = 0.0;
  for (long long j = j0 + tid; j < j1; j += blockDim.x) {
    const long long k0 = cp[j], k1 = cp[j + 1];
    TC dot = (TC)0;
    if (DOT)
      for (long long k = k0; k < k1; ++k) dot += (TC)val[k] * v_s[ri[k]];
    double t0 = 0.0, t1 = 0.0;
    if (MODE == M_ADAT) {
      t0 = (a.cv_esz[0] == 8 ? cv0[j] : (double)static_cast<const float*>(a.cv[0])[j]) * (double)dot;
    } else if (MODE == M_AX) {
      t0 = cv0[j];
    } else if (MODE == M_ATY) {
      a.out_col[0][j] = (double)dot;
    } else if (MODE == M_RESID) {
      const double x = cv0[j], s = cv1[j], c = cv2[j];
      const double rd = (double)dot + s - c;
      const double d2 = x / s;
      a.out_col[0][j] = rd;
      a.out_col[1][j] = d2;
      a.out_colf[j] = (float)d2;
      t0 = x;
      t1 = a.feasible ? (x - sigma_mu / s) : (x - sigma_mu / s - d2 * rd);
      cred0 += rd * rd;
      cred1 += c * x;
    } else if (MODE == M_DIR) {
      const double x = cv0[j], s = cv1[j], v = cv2[j];
      const double rd = a.feasible ? 0.0 : cv3[j];
      const double ds = -rd - (double)dot;
      const double dx = -x + sigma_mu / s - (x / s) * ds - v / s;
      a.out_col[0][j] = dx;
      a.out_col[1][j] = ds;
      cred0 += x * ds + s * dx;
      cred1 += dx * ds;
    }
    if (NACC > 0) {
      const TC tt0 = (TC)t0, tt1 = (TC)t1;
      for (long long k = k0; k < k1; ++k) {
        const int r = ri[k];
        const TC av = (TC)val[k];
        atomicAdd(&u0[r], av * tt0);
        if (NACC > 1) atomicAdd(&u1[r], av * tt1);
      }
    }
  }
  __syncthreads();
  if (NACC > 0) {
    TC* part = static_cast<TC*>(a.partials) + (size_t)blockIdx.x * 2 * a.lda;
    for (int i = tid; i < a.lda; i += blockDim.x) {
      part[i] = u0[i];
      if (NACC > 1) part[a.lda + i] = u1[i];
    }
  }
  if (a.red_partials) {
    const double r0 = block_sum(cred0, red);
    const double r1 = block_sum(cred1, red);
    if (tid == 0) {
      a.red_partials[2 * blockIdx.x] = r0;
      a.red_partials[2 * blockIdx.x + 1] = r1;
    }
  }
  (void)lane;
  if (a.epilogue == E_NONE) return;
  if (tree_reduce<TC>(a, NACC, &s_flag)) stream_epilogue<TC>(a, NACC, red);
}

// A D W for a CSC A: ADW[r][col_b(j)] += sign_b(j) d_j / sqrt(s) a_rj (FP64 atomics;
// adw is zeroed by the caller).
template <typename TV>
__global__ void k_sparse_sketch(const long long* __restrict__ cp, const int* __restrict__ ri,
                                const TV* __restrict__ val, long long n, const double* __restrict__ dvec,
                                int is_d2, uint64_t seed, long long k, int retry, int s_blocks, int wb,
                                double* __restrict__ adw, int w) {
  const double inv_sqrt_s = 1.0 / sqrt((double)s_blocks);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const double d = is_d2 ? sqrt(dvec[j]) : dvec[j];
    const long long k0 = cp[j], k1 = cp[j + 1];
    for (int b = 0; b < s_blocks; ++b) {
      int col;
      float sg;
      cs_entry(seed, k, retry, b, j, wb, &col, &sg);
      const double sc = (double)sg * d * inv_sqrt_s;
      for (long long q = k0; q < k1; ++q) atomicAdd(&adw[(size_t)ri[q] * w + col], (double)val[q] * sc);
    }
  }
}

namespace {
template <typename TV, typename TC, int MODE>
cudaError_t sp_launch(const StreamArgs& a, int grid, cudaStream_t st) {
  const int nvec = (MODE == M_RESID) ? 3 : 2;
  const int smem = nvec * a.lda * (int)sizeof(TC);
  auto k = k_sparse<TV, TC, MODE>;
  cudaError_t e = ensure_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename TV, typename TC>
cudaError_t sp_mode(int mode, const StreamArgs& a, int grid, cudaStream_t st) {
  switch (mode) {
    case M_ADAT: return sp_launch<TV, TC, M_ADAT>(a, grid, st);
    case M_AX: return sp_launch<TV, TC, M_AX>(a, grid, st);
    case M_RESID: return sp_launch<TV, TC, M_RESID>(a, grid, st);
    case M_DIR: return sp_launch<TV, TC, M_DIR>(a, grid, st);
    case M_ATY: return sp_launch<TV, TC, M_ATY>(a, grid, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

int sparse_grid(int num_sms) { return std::min(num_sms * 2, kGroup * kMaxGroups); }

// fp64: FP64 accumulation (double smem vectors), else FP32.
cudaError_t launch_sparse(int dtype, bool fp64, int mode, const StreamArgs& a, int grid,
                          cudaStream_t st) {
  if (dtype == 0) return sp_mode<double, double>(mode, a, grid, st);
  if (fp64) return sp_mode<float, double>(mode, a, grid, st);
  return sp_mode<float, float>(mode, a, grid, st);
}

cudaError_t launch_sparse_sketch(int dtype, const long long* cp, const int* ri, const void* val,
                                 long long n, const double* dvec, int is_d2, uint64_t seed,
                                 long long k, int retry, int s_blocks, int w, double* adw, int m,
                                 int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(adw, 0, sizeof(double) * (size_t)m * w, st);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (dtype == 0)
    k_sparse_sketch<double><<<grid, 256, 0, st>>>(cp, ri, static_cast<const double*>(val), n, dvec,
                                                  is_d2, seed, k, retry, s_blocks, w / s_blocks, adw, w);
  else
    k_sparse_sketch<float><<<grid, 256, 0, st>>>(cp, ri, static_cast<const float*>(val), n, dvec,
                                                 is_d2, seed, k, retry, s_blocks, w / s_blocks, adw, w);
  return cudaGetLastError();
}

}  // namespace lpk
