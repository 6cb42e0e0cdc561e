// Conversions between FP64 n-vectors and the FP32-pair (double-float) form
// read and written by the double-float streaming passes (stream_df.cu).
//
// GB300 executes an FP64 instruction at a small fraction of the FP32 rate,
// and a warp instruction costs the FP64 pipe the same with one active lane as
// with 32.  The per-column formulas of the residual and direction passes
// therefore take their inputs as FP32 pairs, packed here by full warps, and
// their outputs are unpacked here to the FP64 vectors the rest of the
// iteration uses, together with the column sums the epilogues need:
//   residual pass:  sum r_d^2 and c^T x (stopping test, Alg. 3 step 3);
//   direction pass: (x^T ds + s^T dx)/n and dx^T ds / n (the coefficients of
//                   mu(alpha) in the step-length rule, Alg. 2/3).
// Both sums are reduced in a fixed order (per-CTA partials, then one CTA).
#include "internal.h"

namespace lpk {

__global__ void __launch_bounds__(256) k_df_pack(DfPackArgs a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < a.k) {
        const double v = a.src[q][i];
        const float h = (float)v;
        a.dst[q][i] = make_float2(h, (float)(v - (double)h));
      }
    }
  }
}

// mode 0 (residual): out0 = r_d, out1 = d2, outf = fl32(d2); sums r_d^2, c x
// mode 1 (direction): out0 = dx, out1 = ds; sums x ds + s dx, dx ds
__global__ void __launch_bounds__(256) k_df_unpack(DfUnpackArgs a) {
  __shared__ double red[32];
  __shared__ int s_flag;
  double t0 = 0.0, t1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 p0 = a.df0[i], p1 = a.df1[i];
    const double v0 = (double)p0.x + (double)p0.y;
    const double v1 = (double)p1.x + (double)p1.y;
    a.out0[i] = v0;
    a.out1[i] = v1;
    if (a.mode == 0) {
      a.outf[i] = (float)v1;
      t0 = fma(v0, v0, t0);
      t1 = fma(a.c[i], a.x[i], t1);
    } else {
      t0 += a.x[i] * v1 + a.s[i] * v0;
      t1 = fma(v0, v1, t1);
    }
  }
  t0 = block_sum(t0, red);
  t1 = block_sum(t1, red);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = t0;
    a.part[2 * blockIdx.x + 1] = t1;
  }
  if (!last_block_ticket(a.ticket, &s_flag)) return;
  double u0 = 0.0, u1 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    u0 += __ldcg(a.part + 2 * b);
    u1 += __ldcg(a.part + 2 * b + 1);
  }
  u0 = block_sum(u0, red);
  u1 = block_sum(u1, red);
  if (threadIdx.x == 0) {
    if (a.mode == 0) {
      a.sc->rd2 = u0;
      a.sc->cx = u1;
    } else {
      a.sc->c1 = u0 / (double)a.n;
      a.sc->c2 = u1 / (double)a.n;
    }
  }
}

cudaError_t launch_df_pack(const DfPackArgs& a, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((a.n + 255) / 256, (long long)num_sms * 4));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_df_pack<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_df_unpack(const DfUnpackArgs& a, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((a.n + 255) / 256, (long long)num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_df_unpack<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lpk
