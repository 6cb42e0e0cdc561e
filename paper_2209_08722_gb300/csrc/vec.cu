// m-vector and n-vector kernels of the outer iteration:
//   - the preconditioner application z = Q^{-1} r = R^{-1} R^{-T} r through two
//     triangular GEMVs with the explicit inverse of the R factor of (ADW)^T,
//     with the CG / Chebyshev scalar updates fused into the second GEMV's
//     last-CTA epilogue (Algorithm 1 step 3);
//   - (ADW)^T g for the correction vector (eq. compv);
//   - the step lengths of Algorithms 2-3 (first exit from N(gamma), closed-form
//     minimiser of the gap) and the iterate update;
//   - small utilities (dot products, FP32 copies, R extraction, rank check).
// All arithmetic here is FP64.
#include "internal.h"

#include <mutex>
#include <unordered_map>
#include "df.cuh"

namespace lpk {

std::atomic<long long> g_launches{0};

// The dynamic shared-memory limit is a process-wide attribute of a kernel.
// Handles solving different LPs from different host threads launch the same
// kernel with different sizes, so the attribute only ever grows (under a
// lock): lowering it could invalidate another thread's launch in flight.
cudaError_t ensure_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> set;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = set[func];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// ---------------------------------------------------------------------------
// triangular GEMV with a fused epilogue
// ---------------------------------------------------------------------------
enum GemvEpi : int {
  G_NONE = 0,
  G_PCG_INIT = 1,   // rho = r.z, p = z, f_rec = sqrt(rho)
  G_PCG_B = 2,      // rho' = r.z; beta = rho'/rho; p = z + beta p; done if sqrt(rho') <= 0.5 tol
  G_REFRESH = 3,    // true residual: rho' = r.z; converged if sqrt(rho') <= tol; else residual replacement
                    // (INIT and REFRESH kinds: r.z <= 0 with r != 0 sets inner_done = 3)
  G_CHEB_INIT = 4,  // rho = r.z; dir = z / theta; cheb_rho = 1/s1
  G_CHEB_B = 5,     // cheb recurrence on dir; f_rec = sqrt(r.z)
  G_CHEB_REFRESH = 6,  // true residual: converged if sqrt(r.z) <= tol; direction untouched
  G_PCG_B_LAST = 7,    // G_PCG_B on the last step before a refresh: p and rho are left for it
};

struct GemvArgs {
  const double* M;   // m x m, row i contiguous (ld = m)
  int m;
  int lower;         // 1: row i uses columns [0, i]; 0: columns [i, m)
  const double* x;
  double* y;
  int epi;
  int skip_level;    // return immediately if sc->inner_done >= skip_level (0: never)
  double* r;
  double* p;         // CG search direction / Chebyshev update direction
  double* dy;
  DevScalars* sc;
  unsigned* ticket;
  int* err;
  int t_max;
  double* coef;      // G_PCG_B: beta of CG step j stored at coef[2j+1]
  const double* y_add;  // G_NONE: y = y_add + M x when non-null
  const float2* Mdf;    // full M as FP32 pairs (used instead of M when non-null)
};

__global__ void __launch_bounds__(256) k_gemv_tri(const GemvArgs a) {
  __shared__ int s_flag;
  __shared__ __align__(16) double red[32];  // also read as float4 in the epilogue
  pdl_wait();
  pdl_trigger();
  if (a.skip_level > 0 && a.sc->inner_done >= a.skip_level) return;
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = gridDim.x * warps_per_block;
  if (!a.M && !a.Mdf) {
    // identity (no preconditioner): y = x
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.m; i += gridDim.x * blockDim.x)
      a.y[i] = a.y_add ? a.y_add[i] + a.x[i] : a.x[i];
  } else if (a.Mdf) {
    // full rows in double-float on the FP32 pipe: x split into pairs in shared
    // memory once per CTA, each warp one row, FP64 only for the row result
    extern __shared__ float2 xs[];
    // 16 loads per thread in flight at once (m <= 2048 in one round at 128 threads)
    for (int j0 = 0; j0 < a.m; j0 += 16 * (int)blockDim.x) {
      double v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int j = j0 + k * (int)blockDim.x + (int)threadIdx.x;
        v[k] = j < a.m ? a.x[j] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int j = j0 + k * (int)blockDim.x + (int)threadIdx.x;
        const float h = (float)v[k];
        if (j < a.m) xs[j] = make_float2(h, (float)(v[k] - (double)h));
      }
    }
    __syncthreads();
    // (qh + ql)(vh + vl) into (sh, sl): exact product of the high parts plus
    // the cross terms
    auto mac = [](float2 q, float2 v, float& sh, float& sl) {
      const float pr = __fmul_rn(q.x, v.x);
      float e = fmaf(q.x, v.x, -pr);
      e = fmaf(q.x, v.y, e);
      e = fmaf(q.y, v.x, e);
      float t, c;
      two_sum(sh, pr, t, c);
      sh = t;
      sl = __fadd_rn(sl, __fadd_rn(c, e));
    };
    const bool even = (a.m & 1) == 0;  // rows of pairs start 16-byte aligned
    for (int i = gw; i < a.m; i += nw) {
      const float2* row = a.Mdf + (size_t)i * a.m;
      float sh[2] = {0.0f, 0.0f}, sl[2] = {0.0f, 0.0f};
      if (even) {
        // 16-byte loads of two adjacent entries, 8 per lane in flight at once
        // (the row loads are the latency)
        const float4* row4 = reinterpret_cast<const float4*>(row);
        const int m2 = a.m >> 1;
        const float4* xs4 = reinterpret_cast<const float4*>(xs);
        int j0 = 0;
        for (; j0 + 8 * 32 <= m2; j0 += 8 * 32) {  // whole chunks: no bounds checks
          float4 q[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) q[k] = __ldg(row4 + j0 + k * 32 + lane);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float4 v = xs4[j0 + k * 32 + lane];
            mac(make_float2(q[k].x, q[k].y), make_float2(v.x, v.y), sh[0], sl[0]);
            mac(make_float2(q[k].z, q[k].w), make_float2(v.z, v.w), sh[1], sl[1]);
          }
        }
        for (int j = j0 + lane; j < m2; j += 32) {  // the ragged end
          const float4 q = __ldg(row4 + j), v = xs4[j];
          mac(make_float2(q.x, q.y), make_float2(v.x, v.y), sh[0], sl[0]);
          mac(make_float2(q.z, q.w), make_float2(v.z, v.w), sh[1], sl[1]);
        }
      } else {
        for (int j0 = 0; j0 < a.m; j0 += 8 * 32) {
          float2 q[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int j = j0 + k * 32 + lane;
            q[k] = j < a.m ? __ldg(row + j) : make_float2(0.0f, 0.0f);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int j = j0 + k * 32 + lane;
            const float2 v = j < a.m ? xs[j] : make_float2(0.0f, 0.0f);
            mac(q[k], v, sh[k & 1], sl[k & 1]);
          }
        }
      }
      df_add(sh[0], sl[0], sh[1], sl[1]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh[0], o);
        const float ol = __shfl_xor_sync(0xffffffffu, sl[0], o);
        df_add(sh[0], sl[0], oh, ol);
      }
      if (lane == 0) {
        const double acc = (double)sh[0] + (double)sl[0];
        a.y[i] = a.y_add ? a.y_add[i] + acc : acc;
      }
    }
  } else
  for (int i = gw; i < a.m; i += nw) {
    // lower == 1: columns [0, i]; 0: [i, m); 2: the full row
    const int lo = a.lower ? 0 : i;
    const int hi = a.lower == 1 ? i + 1 : a.m;
    const double* row = a.M + (size_t)i * a.m;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    int j = lo + lane;
    for (; j + 96 < hi; j += 128) {
      acc0 = fma(row[j], a.x[j], acc0);
      acc1 = fma(row[j + 32], a.x[j + 32], acc1);
      acc2 = fma(row[j + 64], a.x[j + 64], acc2);
      acc3 = fma(row[j + 96], a.x[j + 96], acc3);
    }
    for (; j < hi; j += 32) acc0 = fma(row[j], a.x[j], acc0);
    double acc = warp_sum((acc0 + acc1) + (acc2 + acc3));
    if (lane == 0) a.y[i] = a.y_add ? a.y_add[i] + acc : acc;
  }
  if (a.epi == G_NONE) return;
  if (!last_block_ticket(a.ticket, &s_flag)) return;
  // ---- epilogue (one CTA): m-vector CG / Chebyshev updates ----
  // r^T z and r^T r: FP64 per thread, then reduced as FP32 pairs on the FP32
  // pipe (an FP64 warp instruction costs GB300's FP64 unit about 16 cycles);
  // the scalar logic runs in thread 0, which broadcasts the coefficients of the
  // one vector update p = c_z z + c_p p.
  DevScalars* sc = a.sc;
  const double* z = a.y;
  __shared__ double s_coef[3];  // c_z, c_p, update flag
  double rz = 0.0, rr = 0.0;
  for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
    const double ri = a.r[i];
    rz = fma(ri, __ldcg(z + i), rz);
    rr = fma(ri, ri, rr);
  }
  {
    float zh = (float)rz, zl = (float)(rz - (double)(float)rz);
    float qh = (float)rr, ql = (float)(rr - (double)(float)rr);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float a0 = __shfl_xor_sync(0xffffffffu, zh, off), a1 = __shfl_xor_sync(0xffffffffu, zl, off);
      const float b0 = __shfl_xor_sync(0xffffffffu, qh, off), b1 = __shfl_xor_sync(0xffffffffu, ql, off);
      df_add(zh, zl, a0, a1);
      df_add(qh, ql, b0, b1);
    }
    float4* redf = reinterpret_cast<float4*>(red);  // 32 doubles = 16 float4
    const int nwb = (int)(blockDim.x + 31) / 32;    // <= 8 (256 threads)
    if (lane == 0) redf[threadIdx.x >> 5] = make_float4(zh, zl, qh, ql);
    __syncthreads();
    if (threadIdx.x == 0) {
      float sh = 0.0f, sl = 0.0f, th = 0.0f, tl = 0.0f;
      for (int w = 0; w < nwb; ++w) {
        df_add(sh, sl, redf[w].x, redf[w].y);
        df_add(th, tl, redf[w].z, redf[w].w);
      }
      rz = (double)sh + (double)sl;
      rr = (double)th + (double)tl;
      double cz = 0.0, cp = 0.0;
      bool upd = false;
      const double f = sqrt(fmax(rz, 0.0));
      // r^T Q^{-1} r <= 0 with r != 0: the stored Q^{-1} has lost definiteness
      // (rounding), so ||f|| means nothing; the host refactors (inner_done = 3)
      const bool indefinite = rz <= 0.0 && rr > 0.0;
      if (!isfinite(rz)) {
        atomicExch(a.err, ERR_NUMERICAL);
      } else if (indefinite && (a.epi == G_PCG_INIT || a.epi == G_REFRESH || a.epi == G_CHEB_INIT ||
                                a.epi == G_CHEB_REFRESH)) {
        sc->f_true = 0.0;
        sc->inner_done = 3;
      } else if (a.epi == G_PCG_INIT) {
        cz = 1.0;
        upd = true;
        sc->rho = rz;
        sc->rho0 = rz;
        sc->f_rec = f;
        sc->f_true = f;
        sc->inner_done = (f <= sc->tol_f) ? 2 : 0;
      } else if (a.epi == G_PCG_B || a.epi == G_PCG_B_LAST) {
        // CG step k: beta_k = rho_{k+1} / rho_k, p_{k+1} = z + beta_k p_k.  The
        // last step before a refresh (and a step that stops) leaves p_k and
        // rho_k in place: the refresh replaces r and z by their true values and
        // makes this direction update itself, once (residual replacement).
        const double beta = rz / sc->rho;
        const bool stop = f <= 0.5 * sc->tol_f;
        const bool defer = stop || a.epi == G_PCG_B_LAST || sc->inner_iters + 1 >= a.t_max;
        if (!defer) {
          cz = 1.0;
          cp = beta;
          upd = true;
          sc->rho = rz;
          if (a.coef && sc->inner_iters < 1024) a.coef[2 * sc->inner_iters + 1] = beta;
        }
        sc->f_rec = f;
        sc->inner_iters += 1;
        if (stop || sc->inner_iters >= a.t_max) sc->inner_done = 1;
      } else if (a.epi == G_REFRESH) {
        // true residual r = p - M dy, z = Q^{-1} r: converged if sqrt(r.z) <= tol;
        // else p = z + (r.z / rho_k) p_k, or p = z (restart) when the recursion
        // drifted far from the FP64 residual (FP32 products).
        double beta = rz / sc->rho;
        const bool stop = f <= sc->tol_f;
        if (f > 4.0 * sc->f_rec) beta = 0.0;
        if (!stop) {
          cz = 1.0;
          cp = beta;
          upd = true;
        }
        sc->rho = rz;
        const int j = sc->inner_iters - 1;  // the deferred step's coefficient
        if (a.coef && j >= 0 && j < 1024) a.coef[2 * j + 1] = beta;
        sc->f_true = f;
        sc->inner_done = stop ? 2 : 0;
      } else if (a.epi == G_CHEB_INIT) {
        const double theta = 0.5 * (sc->lam_max + sc->lam_min);
        const double delta = 0.5 * (sc->lam_max - sc->lam_min);
        cz = 1.0 / theta;
        upd = true;
        sc->cheb_rho = delta / theta;
        sc->rho0 = rz;
        sc->f_rec = f;
        sc->f_true = f;
        sc->inner_done = (f <= sc->tol_f) ? 2 : 0;
      } else if (a.epi == G_CHEB_REFRESH) {
        sc->f_true = f;
        sc->inner_done = (f <= sc->tol_f) ? 2 : 0;
      } else if (a.epi == G_CHEB_B) {
        const double theta = 0.5 * (sc->lam_max + sc->lam_min);
        const double delta = 0.5 * (sc->lam_max - sc->lam_min);
        const double s1 = theta / delta;
        const double rho = sc->cheb_rho;
        const double rho_new = 1.0 / (2.0 * s1 - rho);
        cz = 2.0 * rho_new / delta;
        cp = rho_new * rho;
        upd = true;
        sc->cheb_rho = rho_new;
        sc->f_rec = f;
        sc->inner_iters += 1;
        if (f <= 0.5 * sc->tol_f || sc->inner_iters >= a.t_max) sc->inner_done = 1;
      }
      s_coef[0] = cz;
      s_coef[1] = cp;
      s_coef[2] = upd ? 1.0 : 0.0;
    }
  }
  __syncthreads();  // every thread of the CTA reaches this one barrier
  if (s_coef[2] != 0.0) {
    const double cz = s_coef[0], cp = s_coef[1];
    for (int i = threadIdx.x; i < a.m; i += blockDim.x) a.p[i] = fma(cp, a.p[i], cz * __ldcg(z + i));
  }
}

cudaError_t launch_gemv_tri(const double* M, int m, int lower, const double* x, double* y, int epi,
                            int skip_level, double* r, double* p, double* dy, DevScalars* sc,
                            unsigned* ticket, int* err, int t_max, double* coef, int num_sms,
                            cudaStream_t st, const double* y_add, const float2* Mdf, bool pdl) {
  if ((Mdf || !M) && lower != 2) return cudaErrorInvalidValue;
  GemvArgs a{M, m, lower, x, y, epi, skip_level, r, p, dy, sc, ticket, err, t_max, coef, y_add, Mdf};
  const int warps = Mdf ? 4 : 8;
  int grid = (m + warps - 1) / warps;
  grid = std::max(1, std::min(grid, num_sms * 4));
  const size_t smem = Mdf ? (size_t)m * sizeof(float2) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem((const void*)k_gemv_tri, (int)smem);
    if (e != cudaSuccess) return e;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const cudaError_t e = launch_maybe_pdl(k_gemv_tri, dim3(grid), dim3(warps * 32), smem, st, pdl, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// y_i = alpha y0_i + beta (M x)_i for a rows x cols row-major M (warp per row)
__global__ void __launch_bounds__(256) k_gemv_rows(const double* __restrict__ M, int rows, int cols,
                                                   const double* __restrict__ x,
                                                   const double* __restrict__ y0, double alpha,
                                                   double beta, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int i = gw; i < rows; i += nw) {
    const double* row = M + (size_t)i * cols;
    double acc = 0.0;
    for (int j = lane; j < cols; j += 32) acc = fma(row[j], x[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[i] = (y0 ? alpha * y0[i] : 0.0) + beta * acc;
  }
}

cudaError_t launch_gemv_rows(const double* M, int rows, int cols, const double* x, const double* y0,
                             double alpha, double beta, double* y, int num_sms, cudaStream_t st) {
  const int grid = std::max(1, std::min((rows + 7) / 8, num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_gemv_rows<<<grid, 256, 0, st>>>(M, rows, cols, x, y0, alpha, beta, y);
  return cudaGetLastError();
}

// Chebyshev / residual helpers on m-vectors (one CTA)
__global__ void k_cheb_pre(int m, double* dy, const double* dir, DevScalars* sc) {
  if (sc->inner_done >= 1) return;
  for (int i = threadIdx.x; i < m; i += blockDim.x) dy[i] += dir[i];
}

cudaError_t launch_cheb_pre(int m, double* dy, const double* dir, DevScalars* sc, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_cheb_pre<<<1, 256, 0, st>>>(m, dy, dir, sc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// u = (ADW)^T g, adw row-major m x w: partial sums over row slices, then a sum
// ---------------------------------------------------------------------------
__global__ void k_adwt_partial(const double* __restrict__ adw, int m, int w,
                               const double* __restrict__ g, int rows_per, double* part) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = blockIdx.y * rows_per;
  const int i1 = min(m, i0 + rows_per);
  if (k >= w) return;
  double acc = 0.0;
  for (int i = i0; i < i1; ++i) acc = fma(adw[(size_t)i * w + k], g[i], acc);
  part[(size_t)blockIdx.y * w + k] = acc;
}

__global__ void k_sum_rows(const double* __restrict__ part, int nparts, int w, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= w) return;
  double acc = 0.0;
  for (int q = 0; q < nparts; ++q) acc += part[(size_t)q * w + k];
  out[k] = acc;
}

cudaError_t launch_adwt(const double* adw, int m, int w, const double* g, double* part, int max_parts,
                        double* out, int num_sms, cudaStream_t st) {
  const int bx = (w + 255) / 256;
  int ny = std::max(1, std::min(max_parts, (num_sms * 2 + bx - 1) / bx));
  ny = std::min(ny, m);
  const int rows_per = (m + ny - 1) / ny;
  ny = (m + rows_per - 1) / rows_per;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_adwt_partial<<<dim3(bx, ny), 256, 0, st>>>(adw, m, w, g, rows_per, part);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_sum_rows<<<bx, 256, 0, st>>>(part, ny, w, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dot over n with a last-CTA finish: *out = scale * sum x_i y_i
// ---------------------------------------------------------------------------
__global__ void k_dot(long long n, const double* __restrict__ x, const double* __restrict__ y,
                      double scale, double* part, unsigned* ticket, double* out) {
  __shared__ double red[32];
  __shared__ int s_flag;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (!last_block_ticket(ticket, &s_flag)) return;
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + b);
    *out = scale * t;
  }
}

cudaError_t launch_dot(long long n, const double* x, const double* y, double scale, double* part,
                       unsigned* ticket, double* out, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_dot<<<grid, 256, 0, st>>>(n, x, y, scale, part, ticket, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// step lengths (Algorithm 2 steps 5-6, Algorithm 3 steps 6-7)
// ---------------------------------------------------------------------------
// First alpha > 0 where g(t) = qa t^2 + qb t + qc crosses from >= 0 to < 0;
// +inf if it never does; 0 if g < 0 on all of (0, inf).
__device__ __forceinline__ double first_exit(double qa, double qb, double qc) {
  if (qa == 0.0) {
    if (qb < 0.0) return fmax(-qc / qb, 0.0);
    return INFINITY;
  }
  const double disc = qb * qb - 4.0 * qa * qc;
  if (disc < 0.0) return qa < 0.0 ? 0.0 : INFINITY;
  const double sq = sqrt(disc);
  const double qq = -0.5 * (qb + (qb >= 0.0 ? sq : -sq));
  double r1 = 0.0, r2 = 0.0;
  if (qq != 0.0) {
    r1 = qq / qa;
    r2 = qc / qq;
  }
  const double lo = fmin(r1, r2), hi = fmax(r1, r2);
  if (qa > 0.0) return lo > 0.0 ? lo : INFINITY;
  return hi > 0.0 ? hi : 0.0;
}

struct StepArgs {
  long long n;
  const double *x, *s, *dx, *ds;
  double gamma;
  int feasible;
  double res_ratio;  // ||r|| / ||r^0||
  double mu0;
  double* part;      // [grid][2]: min over elements of the N(gamma) exit and the positivity exit
  unsigned* ticket;
  DevScalars* sc;
};

__global__ void __launch_bounds__(256) k_step(const StepArgs a) {
  __shared__ double red[32];
  __shared__ int s_flag;
  const double mu = a.sc->mu;
  const double c1 = a.sc->c1, c2 = a.sc->c2;
  const double g = 1.0 - a.gamma;
  double ex = INFINITY, pos = INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    const double x = a.x[i], s = a.s[i], dx = a.dx[i], ds = a.ds[i];
    ex = fmin(ex, first_exit(dx * ds - g * c2, x * ds + s * dx - g * c1, x * s - g * mu));
    if (dx < 0.0) pos = fmin(pos, -x / dx);
    if (ds < 0.0) pos = fmin(pos, -s / ds);
  }
  ex = block_min(ex, red);
  pos = block_min(pos, red);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = ex;
    a.part[2 * blockIdx.x + 1] = pos;
  }
  if (!last_block_ticket(a.ticket, &s_flag)) return;
  if (threadIdx.x != 0) return;
  double e = INFINITY, p = INFINITY;
  for (int b = 0; b < (int)gridDim.x; ++b) {
    e = fmin(e, __ldcg(a.part + 2 * b));
    p = fmin(p, __ldcg(a.part + 2 * b + 1));
  }
  double alpha = fmin(1.0, e);
  alpha = fmin(alpha, first_exit(c2, c1, mu));  // mu(alpha) > 0
  if (!a.feasible)
    alpha = fmin(alpha, first_exit(c2 / a.mu0, c1 / a.mu0 + a.res_ratio, mu / a.mu0 - a.res_ratio));
  if (p <= alpha) alpha = p * (1.0 - 1e-12);
  const double amax = fmax(alpha, 0.0);
  double abar = amax;
  if (c2 > 0.0) abar = fmin(fmax(-c1 / (2.0 * c2), 0.0), amax);
  a.sc->alpha_max = amax;
  a.sc->alpha_bar = abar;
}

cudaError_t launch_step(long long n, const double* x, const double* s, const double* dx,
                        const double* ds, double gamma, int feasible, double res_ratio, double mu0,
                        double* part, unsigned* ticket, DevScalars* sc, int num_sms,
                        cudaStream_t st) {
  StepArgs a{n, x, s, dx, ds, gamma, feasible, res_ratio, mu0, part, ticket, sc};
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_step<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// sc->alpha_aff = min(1, min_i {-x_i/dx_i : dx_i < 0}, min_i {-s_i/ds_i : ds_i < 0})
__global__ void __launch_bounds__(256) k_pos_step(long long n, const double* __restrict__ x,
                                                  const double* __restrict__ s, const double* __restrict__ dx,
                                                  const double* __restrict__ ds, double* part, unsigned* ticket,
                                                  DevScalars* sc) {
  __shared__ double red[32];
  __shared__ int s_flag;
  double pos = 1.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (dx[i] < 0.0) pos = fmin(pos, -x[i] / dx[i]);
    if (ds[i] < 0.0) pos = fmin(pos, -s[i] / ds[i]);
  }
  pos = block_min(pos, red);
  if (threadIdx.x == 0) part[blockIdx.x] = pos;
  if (!last_block_ticket(ticket, &s_flag)) return;
  double p = 1.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) p = fmin(p, __ldcg(part + b));
  p = block_min(p, red);
  if (threadIdx.x == 0) sc->alpha_aff = p;
}

cudaError_t launch_pos_step(long long n, const double* x, const double* s, const double* dx,
                            const double* ds, double* part, unsigned* ticket, DevScalars* sc, int num_sms,
                            cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_pos_step<<<grid, 256, 0, st>>>(n, x, s, dx, ds, part, ticket, sc);
  return cudaGetLastError();
}

// warm-start features X = [dy_prev / |u|, u / |u|, log10(mu) / 10 * 1] (3m, FP32)
__global__ void k_ws_features(int m, const double* __restrict__ dy_prev, int have_prev,
                              const double* __restrict__ u, const DevScalars* sc, float* __restrict__ X) {
  const double inv = sc->pad[0] > 0.0 ? 1.0 / sqrt(sc->pad[0]) : 0.0;  // 1 / |u|
  const float lm = (float)(log10(fmax(sc->mu, 1e-300)) / 10.0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    X[i] = have_prev ? (float)(dy_prev[i] * inv) : 0.0f;
    X[m + i] = (float)(u[i] * inv);
    X[2 * m + i] = lm;
  }
}

// dir 0: out = |u| * Y (FP32 -> FP64);  dir 1: Yf = in / |u| (FP64 -> FP32)
__global__ void k_ws_scale(int m, int dir, const float* __restrict__ yf, const double* __restrict__ in,
                           const DevScalars* sc, double* __restrict__ out, float* __restrict__ of) {
  const double su = sqrt(fmax(sc->pad[0], 0.0));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (dir == 0) out[i] = su * (double)yf[i];
    else of[i] = su > 0.0 ? (float)(in[i] / su) : 0.0f;
  }
}

cudaError_t launch_ws_features(int m, const double* dy_prev, int have_prev, const double* u,
                               const DevScalars* sc, float* X, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_ws_features<<<(m + 255) / 256, 256, 0, st>>>(m, dy_prev, have_prev, u, sc, X);
  return cudaGetLastError();
}

cudaError_t launch_ws_scale(int m, int dir, const float* yf, const double* in, const DevScalars* sc,
                            double* out, float* of, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_ws_scale<<<(m + 255) / 256, 256, 0, st>>>(m, dir, yf, in, sc, out, of);
  return cudaGetLastError();
}

// x += a dx, s += a ds (n), y += a dy (m); sc->mu = x^T s / n afterwards
__global__ void k_update(long long n, int m, double* x, double* s, double* y, const double* dx,
                         const double* ds, const double* dy, DevScalars* sc, double* part,
                         unsigned* ticket) {
  __shared__ double red[32];
  __shared__ int s_flag;
  const double al = sc->alpha_bar;
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long i = t0; i < n; i += stride) {
    const double xi = x[i] + al * dx[i];
    const double si = s[i] + al * ds[i];
    x[i] = xi;
    s[i] = si;
    acc = fma(xi, si, acc);
  }
  for (long long i = t0; i < m; i += stride) y[i] += al * dy[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (!last_block_ticket(ticket, &s_flag)) return;
  // fixed-order block-parallel sum of the partials
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(part + b);
  t = block_sum(t, red);
  if (threadIdx.x == 0) {
    sc->xs_next = t;
    sc->mu = t / (double)n;
  }
}

cudaError_t launch_update(long long n, int m, double* x, double* s, double* y, const double* dx,
                          const double* ds, const double* dy, DevScalars* sc, double* part,
                          unsigned* ticket, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_update<<<grid, 256, 0, st>>>(n, m, x, s, y, dx, ds, dy, sc, part, ticket);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// utilities
// ---------------------------------------------------------------------------
// out = alpha x + beta y
__global__ void k_axpby(long long n, double alpha, const double* __restrict__ x, double beta,
                        const double* __restrict__ y, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = alpha * x[i] + beta * y[i];
}

cudaError_t launch_axpby(long long n, double alpha, const double* x, double beta, const double* y,
                         double* out, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_axpby<<<grid, 256, 0, st>>>(n, alpha, x, beta, y, out);
  return cudaGetLastError();
}

__global__ void k_fill(long long n, double* x, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

cudaError_t launch_fill(long long n, double* x, double v, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_fill<<<grid, 256, 0, st>>>(n, x, v);
  return cudaGetLastError();
}

// Health check of the bounded waits: the wait every pipeline uses, on a
// barrier whose phase completes only if this thread arrives on it first.
__global__ void k_wait_probe(int* err, long long limit, int complete) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (complete) mbar_arrive(&bar);
    mbar_wait_for(&bar, 0u, err, limit);
  }
}

cudaError_t launch_wait_probe(int* err, long long limit, int complete, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_wait_probe<<<1, 32, 0, st>>>(err, limit, complete);
  return cudaGetLastError();
}

// *out = min_i x_i y_i
__global__ void k_min_prod(long long n, const double* __restrict__ x, const double* __restrict__ y,
                           double* part, unsigned* ticket, double* out) {
  __shared__ double red[32];
  __shared__ int s_flag;
  double mn = INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    mn = fmin(mn, x[i] * y[i]);
  mn = block_min(mn, red);
  if (threadIdx.x == 0) part[blockIdx.x] = mn;
  if (!last_block_ticket(ticket, &s_flag)) return;
  if (threadIdx.x == 0) {
    double t = INFINITY;
    for (int b = 0; b < (int)gridDim.x; ++b) t = fmin(t, __ldcg(part + b));
    *out = t;
  }
}

cudaError_t launch_min_prod(long long n, const double* x, const double* y, double* part,
                            unsigned* ticket, double* out, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_min_prod<<<grid, 256, 0, st>>>(n, x, y, part, ticket, out);
  return cudaGetLastError();
}
__global__ void k_to_f32(long long n, const double* __restrict__ x, float* __restrict__ y, int square) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    y[i] = (float)(square ? v * v : v);
  }
}

__global__ void k_square(long long n, const double* __restrict__ x, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * x[i];
}

cudaError_t launch_to_f32(long long n, const double* x, float* y, int square, int num_sms,
                          cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_to_f32<<<grid, 256, 0, st>>>(n, x, y, square);
  return cudaGetLastError();
}

cudaError_t launch_square(long long n, const double* x, double* y, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_square<<<grid, 256, 0, st>>>(n, x, y);
  return cudaGetLastError();
}

// R (upper m x m of a column-major w x m array, ld = w) -> dst column-major m x m,
// zero below the diagonal; diagonal extremes into sc for the rank check.
__global__ void k_extract_r(const double* __restrict__ qr, int w, int m, double* __restrict__ dst) {
  const long long total = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / m), i = (int)(e % m);  // column j, row i
    dst[e] = (i <= j) ? qr[(size_t)j * w + i] : 0.0;
  }
}

__global__ void k_diag_range(const double* __restrict__ r, int m, DevScalars* sc, double rank_tol) {
  __shared__ double red[32];
  double mn = INFINITY, mx = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double d = fabs(r[(size_t)i * m + i]);
    mn = fmin(mn, d);
    mx = fmax(mx, d);
  }
  mn = block_min(mn, red);
  mx = -block_min(-mx, red);
  if (threadIdx.x == 0) {
    sc->diag_min = mn;
    sc->diag_max = mx;
    sc->rank_bad = (!(mn > rank_tol * mx) || !isfinite(mx)) ? 1 : 0;
  }
}

// mirror the upper triangle of a column-major m x m matrix into its lower one
__global__ void k_symmetrize(double* __restrict__ a, int m) {
  const long long total = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / m), i = (int)(e % m);  // column j, row i
    if (i > j) a[e] = a[(size_t)i * m + j];
  }
}

__global__ void k_transpose(const double* __restrict__ src, int m, double* __restrict__ dst) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = by + k, c = bx + threadIdx.x;
    if (r < m && c < m) tile[k][threadIdx.x] = src[(size_t)r * m + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = bx + k, c = by + threadIdx.x;
    if (r < m && c < m) dst[(size_t)r * m + c] = tile[threadIdx.x][k];
  }
}

cudaError_t launch_factor_utils(int which, const double* a, int w, int m, double* b, DevScalars* sc,
                                double rank_tol, int num_sms, cudaStream_t st) {
  if (which == 0) {
    const long long total = (long long)m * m;
    const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, num_sms * 4));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_extract_r<<<grid, 256, 0, st>>>(a, w, m, b);
  } else if (which == 1) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_diag_range<<<1, 256, 0, st>>>(a, m, sc, rank_tol);
  } else if (which == 3) {
    const long long total = (long long)m * m;
    const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, num_sms * 4));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_symmetrize<<<grid, 256, 0, st>>>(b, m);
  } else {
    dim3 grid((m + 31) / 32, (m + 31) / 32);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(a, m, b);
  }
  return cudaGetLastError();
}

}  // namespace lpk
