// Shared device helpers for the sm_103a kernels of the sketched IPM.
//
// - PTX wrappers for mbarrier and the 1-D bulk async copy (cp.async.bulk),
//   used to stream column tiles of A from HBM into shared memory.
// - Bounded waits: every spin on an mbarrier gives up after ~1 s of clock64
//   cycles, records LPK_ERR_TIMEOUT in the device status word and returns.
// - SplitMix64 counter-based generator for the CountSketch W.
// - Device-side scalar block shared by the solver kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lpk {

constexpr int kThreads = 256;          // threads per CTA for the streaming kernels
constexpr int kWarps = kThreads / 32;
constexpr int kConsumerWarps = 16;     // consumer warps of the fused product kernel
constexpr int kFusedThreads = (kConsumerWarps + 1) * 32;  // + one producer warp
constexpr int kMaxStages = 4;
constexpr int kGroup = 8;              // CTAs per first-level reduction group
constexpr int kMaxGroups = 64;         // group tickets; slot kMaxGroups is the global one
constexpr int kMaxColVecs = 4;         // per-column input vectors staged with a tile
constexpr long long kSpinCycles = 1LL << 31;

// device status word values (DevScalars::err)
enum : int { ERR_NONE = 0, ERR_TIMEOUT = 1, ERR_NUMERICAL = 2 };

// ---------------------------------------------------------------------------
// scalars living in device memory, written and read by kernels
// ---------------------------------------------------------------------------
struct DevScalars {
  // outer iteration
  double mu;          // x^T s / n of the current iterate
  double cx, by;      // c^T x, b^T y
  double rp2, rd2;    // ||r_p||^2, ||r_d||^2
  double c1, c2;      // (x^T ds + s^T dx)/n, dx^T ds / n
  double alpha_max, alpha_bar;
  double xs_next;     // sum x_i s_i after the update (next mu * n)
  // inner solve (PCG on the normal equations)
  double rho;         // r^T z of the current residual
  double rho0;        // r^T z at the start (||f^(0)||^2)
  double pq;          // p^T q
  double tol_f;       // stopping level for ||f||
  double f_true;      // last FP64 ||f|| (true residual)
  double f_rec;       // last recursive ||f||
  double dot_tmp;
  double cheb_rho;    // Chebyshev recurrence scalar
  double lam_min, lam_max;
  int inner_done;     // 1: recursive residual small, 2: true residual converged,
                      // 3: r^T Q^{-1} r <= 0 (indefinite stored Q^{-1})
  int inner_iters;    // iterations taken by the inner solver
  int rank_bad;       // sketch factor rank check failed
  int err;            // ERR_* (sticky)
  double diag_min, diag_max;
  double alpha_aff;   // largest positivity-keeping step of the affine direction (<= 1)
  double pad[4];
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel of its stream is still
// running; pdl_wait() returns once that kernel has completed and its writes are
// visible (at once when there is no such dependency), and pdl_trigger() lets
// the next such kernel start launching.  Both are called first thing, before
// any read of a previous kernel's results.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The same copy with an L2 "evict first" hint: for data read once per pass
// (the columns of A), so that streaming it through L2 does not push out what
// the next kernels reuse (the preconditioner, the per-column vectors).
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
      "%4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity`: false (and err = ERR_TIMEOUT) once `limit`
// clock64 cycles have passed without the phase completing.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, int* err, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicExch(err, ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// The wait every pipeline uses: gives up after kSpinCycles (~1 s).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  return mbar_wait_for(bar, parity, err, kSpinCycles);
}

// ---------------------------------------------------------------------------
// warp / block reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the block; every thread gets the result.  `buf` >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* buf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) buf[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? buf[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) buf[0] = t;
  __syncthreads();
  double r = buf[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_min(double v, double* buf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) buf[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? buf[threadIdx.x] : INFINITY;
  if (wid == 0) t = warp_min(t);
  if (threadIdx.x == 0) buf[0] = t;
  __syncthreads();
  double r = buf[0];
  __syncthreads();
  return r;
}

// Ticket for the "last CTA finishes" pattern.  Call after this CTA's partial
// results are stored; returns true in exactly one CTA (the last), in which all
// other CTAs' stores are visible.  Resets the counter for the next launch.
__device__ __forceinline__ bool last_block_ticket(unsigned* ticket, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    const bool last = (t == gridDim.x * gridDim.y - 1);
    if (last) *ticket = 0u;
    *s_flag = last ? 1 : 0;
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based generator:
// output t (t >= 1) of the stream seeded with S is mix64(S + t * GAMMA).
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kMaxRetry = 16;
constexpr int kMaxBlocks = 16;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// draw at counter `ctr` = output ctr+1 of the stream seeded with `seed`
__host__ __device__ __forceinline__ uint64_t sm64_draw(uint64_t seed, uint64_t ctr) {
  return mix64(seed + (ctr + 1ull) * kGamma);
}

// CountSketch entry of row i in block b for outer iteration k, redraw r:
// column b*wb + ((hi32 * wb) >> 32), sign +1 if the low bit is 0.
__host__ __device__ __forceinline__ uint64_t cs_counter(long long k, int retry, int block,
                                                        long long i) {
  const uint64_t hi = ((uint64_t)((k * kMaxRetry + retry) * kMaxBlocks + block)) << 40;
  return hi + (uint64_t)i;
}

__device__ __forceinline__ void cs_entry(uint64_t seed, long long k, int retry, int block,
                                         long long i, int wb, int* col, float* sign) {
  const uint64_t v = sm64_draw(seed, cs_counter(k, retry, block, i));
  const uint32_t h = (uint32_t)(((v >> 32) * (uint64_t)wb) >> 32);
  *col = block * wb + (int)h;
  *sign = (v & 1ull) ? -1.0f : 1.0f;
}

// ---------------------------------------------------------------------------
// element loads of 16-byte vectors from shared memory, converted to TC
// ---------------------------------------------------------------------------
struct bf16raw { uint16_t b; };

template <typename TA> struct VecOf;
template <> struct VecOf<double> { static constexpr int N = 2; };
template <> struct VecOf<float> { static constexpr int N = 4; };
template <> struct VecOf<bf16raw> { static constexpr int N = 8; };

template <typename TC>
__device__ __forceinline__ void ld16(const double* p, TC* o) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = (TC)v.x;
  o[1] = (TC)v.y;
}
template <typename TC>
__device__ __forceinline__ void ld16(const float* p, TC* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = (TC)v.x;
  o[1] = (TC)v.y;
  o[2] = (TC)v.z;
  o[3] = (TC)v.w;
}
template <typename TC>
__device__ __forceinline__ void ld16(const bf16raw* p, TC* o) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[2 * q] = (TC)__uint_as_float(w[q] << 16);
    o[2 * q + 1] = (TC)__uint_as_float(w[q] & 0xFFFF0000u);
  }
}

}  // namespace lpk
