// Column passes over a sparse A in CSC form (col_ptr int64, row_idx int32,
// values FP32 or FP64): the product A diag(d2) A^T v, the residual /
// right-hand-side pass, the direction pass and the CountSketch A D W.
//
// The passes run in a deterministic two-pass form (below): no atomics, so
// sparse solves are bitwise reproducible.  The CountSketch of a CSC A is in
// sketch.cu (k_sp_bucket, reproducible); k_sparse_sketch here is its
// FP64-atomic fallback for buckets or sizes the bucket lists cannot hold.
#include "internal.h"
#include "stream_dev.cuh"

namespace lpk {

// ---------------------------------------------------------------------------
// Deterministic two-pass passes over a sparse A held by columns (CSC) and by
// rows (CSR): the column pass gathers a_j^T v from a shared-memory copy of v
// (thread per column) and forms the per-column scalars t0_j, t1_j and
// outputs; the row pass sums a_ij t_j over each row segment (warp per segment
// of at most kSegNnz entries, so heavy rows split evenly) with t gathered from
// global memory (L2-resident); a one-CTA epilogue adds each row's segments in
// order and runs the mode's epilogue.  No atomics: the result is the same in
// every run.
// ---------------------------------------------------------------------------
template <typename TV, typename TC, int MODE>
__global__ void __launch_bounds__(256) k_spc(const StreamArgs a) {
  constexpr int NACC = (MODE == M_RESID) ? 2 : ((MODE == M_ADAT || MODE == M_AX) ? 1 : 0);
  constexpr bool DOT = (MODE != M_AX);
  extern __shared__ __align__(16) char smem[];
  TC* v_s = reinterpret_cast<TC*>(smem);
  __shared__ double red[64];
  __shared__ int s_flag;
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;
  const int tid = threadIdx.x;
  const double sigma_mu = a.sigma * a.sc->mu;
  const long long* cp = a.colptr;
  const int* ri = a.rowidx;
  const TV* val = static_cast<const TV*>(a.spval);
  if (DOT)
    for (int i = tid; i < a.lda; i += blockDim.x) v_s[i] = i < a.m ? (TC)a.vin[i] : (TC)0;
  __syncthreads();
  const double* cv0 = static_cast<const double*>(a.cv[0]);
  const double* cv1 = static_cast<const double*>(a.cv[1]);
  const double* cv2 = static_cast<const double*>(a.cv[2]);
  const double* cv3 = static_cast<const double*>(a.cv[3]);
  TC* t0v = static_cast<TC*>(a.tcol);
  TC* t1v = t0v + a.n;
  double cred0 = 0.0, cred1 = 0.0;
  for (long long j = blockIdx.x * (long long)blockDim.x + tid; j < a.n; j += (long long)gridDim.x * blockDim.x) {
    TC dot = (TC)0;
    if (DOT) {
      const long long k0 = cp[j], k1 = cp[j + 1];
      for (long long k = k0; k < k1; ++k) dot += (TC)val[k] * v_s[ri[k]];
    }
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
    if (NACC > 0) t0v[j] = (TC)t0;
    if (NACC > 1) t1v[j] = (TC)t1;
  }
  if (MODE == M_RESID || MODE == M_DIR) {
    // column reductions: per CTA, then the last CTA adds them in CTA order
    const double r0 = block_sum(cred0, red);
    const double r1 = block_sum(cred1, red);
    if (tid == 0) {
      a.red_partials[2 + 2 * blockIdx.x] = r0;
      a.red_partials[3 + 2 * blockIdx.x] = r1;
    }
    if (!last_block_ticket(a.ticket, &s_flag)) return;
    double t0 = 0.0, t1 = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
      t0 += __ldcg(a.red_partials + 2 + 2 * b);
      t1 += __ldcg(a.red_partials + 3 + 2 * b);
    }
    t0 = block_sum(t0, red);
    t1 = block_sum(t1, red);
    if (tid == 0) {
      if (MODE == M_DIR) {
        a.sc->c1 = t0 / (double)a.n;
        a.sc->c2 = t1 / (double)a.n;
      } else {
        a.red_partials[0] = t0;
        a.red_partials[1] = t1;
      }
    }
  }
}

// warp per row segment: the segment's sums of a_ij t0_j (and a_ij t1_j)
template <typename TV, typename TC, int NACC>
__global__ void __launch_bounds__(256) k_spr(const StreamArgs a) {
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const TV* val = static_cast<const TV*>(a.rval);
  const TC* t0v = static_cast<const TC*>(a.tcol);
  const TC* t1v = t0v + a.n;
  for (int sgi = warp; sgi < a.nseg; sgi += nw) {
    const long long k0 = a.seg[2 * sgi], k1 = a.seg[2 * sgi + 1];
    TC s0 = (TC)0, s1 = (TC)0;
    for (long long k = k0 + lane; k < k1; k += 32) {
      const int c = a.colidx[k];
      const TC av = (TC)val[k];
      s0 += av * __ldg(t0v + c);
      if (NACC > 1) s1 += av * __ldg(t1v + c);
    }
    s0 = warp_sum(s0);
    if (NACC > 1) s1 = warp_sum(s1);
    if (lane == 0) {
      a.segsum[2 * sgi] = (double)s0;
      if (NACC > 1) a.segsum[2 * sgi + 1] = (double)s1;
    }
  }
}

// one CTA: each row's segments added in order into the group-sum slots the
// streaming epilogue reads (one group), then that epilogue
template <typename TC, int NACC>
__global__ void __launch_bounds__(1024) k_spe(const StreamArgs a) {
  __shared__ double red[64];
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;
  for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = a.row_seg[i]; q < a.row_seg[i + 1]; ++q) {
      s0 += a.segsum[2 * q];
      if (NACC > 1) s1 += a.segsum[2 * q + 1];
    }
    if constexpr (sizeof(TC) == 4) {
      float2* g = reinterpret_cast<float2*>(a.gpart);
      const float h0 = (float)s0, h1 = (float)s1;
      g[i] = make_float2(h0, (float)(s0 - (double)h0));
      if (NACC > 1) g[a.lda + i] = make_float2(h1, (float)(s1 - (double)h1));
    } else {
      a.gpart[i] = s0;
      if (NACC > 1) a.gpart[a.lda + i] = s1;
    }
  }
  __syncthreads();
  __threadfence_block();
  stream_epilogue<TC>(a, NACC, red);
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

// the grid of a sparse handle's reduction plan (it sizes the handle's buffer of
// per-CTA reduction partials, shared with the dense passes)
int sparse_grid(int num_sms) { return std::min(num_sms * 2, kGroup * kMaxGroups); }

namespace {
template <typename TV, typename TC, int MODE>
cudaError_t sp2_launch(StreamArgs a, int num_sms, cudaStream_t st) {
  constexpr int NACC = (MODE == M_RESID) ? 2 : ((MODE == M_ADAT || MODE == M_AX) ? 1 : 0);
  const int smem = a.lda * (int)sizeof(TC);
  auto kc = k_spc<TV, TC, MODE>;
  cudaError_t e = ensure_smem((const void*)kc, smem);
  if (e != cudaSuccess) return e;
  const int gc = (int)std::max<long long>(1, std::min<long long>((a.n + 255) / 256, (long long)num_sms * 8));
  if (MODE == M_RESID || MODE == M_DIR) a.red_partials = a.segsum + 2 * (size_t)a.nseg;  // [2 + 2 gc]
  g_launches.fetch_add(1, std::memory_order_relaxed);
  kc<<<gc, 256, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || NACC == 0) return e;
  const int gr = std::max(1, std::min((a.nseg + 7) / 8, num_sms * 8));
  g_launches.fetch_add(2, std::memory_order_relaxed);
  k_spr<TV, TC, NACC><<<gr, 256, 0, st>>>(a);
  if (MODE != M_RESID) a.red_partials = nullptr;
  k_spe<TC, NACC><<<1, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename TV, typename TC>
cudaError_t sp2_mode(int mode, const StreamArgs& a, int num_sms, cudaStream_t st) {
  switch (mode) {
    case M_ADAT: return sp2_launch<TV, TC, M_ADAT>(a, num_sms, st);
    case M_AX: return sp2_launch<TV, TC, M_AX>(a, num_sms, st);
    case M_RESID: return sp2_launch<TV, TC, M_RESID>(a, num_sms, st);
    case M_DIR: return sp2_launch<TV, TC, M_DIR>(a, num_sms, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

// the grid size the column pass of the two-pass kernels uses (its column
// reductions take 2 + 2 grid doubles after the segment sums)
int sparse2_col_grid(long long n, int num_sms) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 8));
}

cudaError_t launch_sparse2(int dtype, bool fp64, int mode, const StreamArgs& a, int num_sms, cudaStream_t st) {
  if (dtype == 0) return sp2_mode<double, double>(mode, a, num_sms, st);
  if (fp64) return sp2_mode<float, double>(mode, a, num_sms, st);
  return sp2_mode<float, float>(mode, a, num_sms, st);
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
