// The warm-start model's dense contractions (mlp.cu): a column-major FP32 GEMM
// on the tcgen05 tensor cores, and an FP32 GEMV for single-sample prediction.
//
// GEMM: C (M x N) = op(A) (M x K) * op(B) (K x N), every matrix column-major,
// op = identity or transpose (the three forms the forward and backward passes
// use: NN, NT and TN).  FP32 accuracy from TF32 tensor-core products by
// splitting each operand, x = x_hi + x_lo with x_hi = tf32(x) and
// x_lo = tf32(x - x_hi):  op(A) op(B) ~ A_hi B_hi + A_lo B_hi + A_hi B_lo
// (A_lo B_lo, about 2^-22 relative, is dropped); FP32 accumulation in tensor
// memory.  A CTA owns one 128 x 128 tile of C and runs over all of K in chunks
// of 16: 256 threads load the chunk's op(A) rows and op(B) columns (the next
// chunk is loaded into registers while the current one is staged), split them
// and store the four 128 x 16 operand tiles in shared memory in the K-major
// core-matrix layout; one thread issues the six MMAs (M = N = 128, K = 8) of
// the chunk and commits them to the chunk's mbarrier; two buffers overlap the
// staging with the tensor core.  The FP32 tile is read back with tcgen05.ld
// and stored column-major.  Waits are bounded (a timeout sets the error word)
// and tensor memory is released on every path.
//
// GEMV: y = W x for a column-major W (rows x cols) and one sample; column
// slices of W go to different CTAs (thread per row, coalesced along rows) and
// their partial sums are added in slice order by the bias kernel that follows.
#include "internal.h"
#include "tc.cuh"

namespace lpk {

namespace {

constexpr int G_M = 128;
constexpr int G_N = 128;
constexpr int G_BK = 16;
constexpr int G_THREADS = 256;
constexpr int G_LBO = 128;                  // next core matrix along K
constexpr int G_SBO = (G_BK / 4) * 128;     // next group of 8 rows
constexpr int G_TILE = 128 * G_BK * 4;      // one 128 x 16 FP32 operand tile (8 KB)
constexpr int G_STAGE = 4 * G_TILE;         // A_hi, A_lo, B_hi, B_lo
constexpr int G_SMEM = 2 * G_STAGE + 1024;  // two stages + alignment slack (<= 3 CTAs per SM)

__device__ __forceinline__ int g_core_off(int r, int k4) { return (r >> 3) * G_SBO + k4 * G_LBO + (r & 7) * 16; }

}  // namespace

template <bool TA, bool TB>
__global__ void __launch_bounds__(G_THREADS, 1)
    k_gemm_tf32x3(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B,
                  int ldb, float* __restrict__ C, int ldc, int* err) {
  extern __shared__ char smem_raw[];
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * G_M, j0 = blockIdx.y * G_N;
  const int nchunks = (K + G_BK - 1) / G_BK;
  if (warp == 0) tc_alloc(&tmem_s, G_N);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_s;
  constexpr uint32_t idesc = tc_idesc_tf32(G_M, G_N);

  // staging roles: thread t owns operand row r = t % 128 (a row of op(A) and a
  // column of op(B)) and the k groups g and g + 2 (4 consecutive k each)
  const int r = tid & 127, g = tid >> 7;
  float ra[2][4], rb[2][4];
  auto load_chunk = [&](int kb) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = kb + (g + 2 * h) * 4 + q;
        const int i = i0 + r, j = j0 + r;
        ra[h][q] = (i < M && k < K) ? (TA ? A[(size_t)i * lda + k] : A[(size_t)k * lda + i]) : 0.0f;
        rb[h][q] = (j < N && k < K) ? (TB ? B[(size_t)k * ldb + j] : B[(size_t)j * ldb + k]) : 0.0f;
      }
  };
  if (nchunks > 0) load_chunk(0);
  bool ok = true;
  int issued = 0;
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    char* stage = smem + (size_t)b * G_STAGE;
    if (c >= 2) {  // the MMAs of chunk c - 2 read this buffer
      const bool w_ok = mbar_wait(&bars[b], (uint32_t)(((c - 2) >> 1) & 1), err);
      ok = __syncthreads_and(w_ok && ok) != 0;
      if (!ok) break;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[q] = tc_to_tf32(ra[h][q]);
        al[q] = tc_to_tf32(ra[h][q] - __uint_as_float(ah[q]));
        bh[q] = tc_to_tf32(rb[h][q]);
        bl[q] = tc_to_tf32(rb[h][q] - __uint_as_float(bh[q]));
      }
      const int off = g_core_off(r, g + 2 * h);
      *reinterpret_cast<uint4*>(stage + off) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
      *reinterpret_cast<uint4*>(stage + G_TILE + off) = make_uint4(al[0], al[1], al[2], al[3]);
      *reinterpret_cast<uint4*>(stage + 2 * G_TILE + off) = make_uint4(bh[0], bh[1], bh[2], bh[3]);
      *reinterpret_cast<uint4*>(stage + 3 * G_TILE + off) = make_uint4(bl[0], bl[1], bl[2], bl[3]);
    }
    if (c + 1 < nchunks) load_chunk((c + 1) * G_BK);
    // the generic-proxy stores must be visible to the tensor core
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after_sync();
      const uint32_t s0 = smem_u32(stage);
#pragma unroll
      for (int s = 0; s < G_BK / 8; ++s) {
        const uint32_t koff = (uint32_t)(s * 2 * G_LBO);  // two core matrices per k-step
        const uint64_t a_hi = tc_sdesc(s0 + koff, G_LBO, G_SBO);
        const uint64_t a_lo = tc_sdesc(s0 + G_TILE + koff, G_LBO, G_SBO);
        const uint64_t b_hi = tc_sdesc(s0 + 2 * G_TILE + koff, G_LBO, G_SBO);
        const uint64_t b_lo = tc_sdesc(s0 + 3 * G_TILE + koff, G_LBO, G_SBO);
        tc_mma_tf32(tmem, a_hi, b_hi, idesc, (c > 0 || s > 0) ? 1u : 0u);
        tc_mma_tf32(tmem, a_lo, b_hi, idesc, 1u);
        tc_mma_tf32(tmem, a_hi, b_lo, idesc, 1u);
      }
      tc_commit_to(&bars[b]);
    }
    issued = c + 1;
  }
  // the last commits cover every MMA; waiting on both buffers' last ones
  // leaves no arrive pending
  bool all_ok = ok;
  for (int c = (issued > 2 ? issued - 2 : 0); c < issued; ++c)
    all_ok = mbar_wait(&bars[c & 1], (uint32_t)((c >> 1) & 1), err) && all_ok;
  all_ok = __syncthreads_and(all_ok) != 0;
  tc_fence_after_sync();
  // warp w reads TMEM lanes 32 (w % 4) .. +32 (rows) and column half w / 4
  const int lq = warp & 3, half = warp >> 2;
  const int i = i0 + lq * 32 + lane;
#pragma unroll 1
  for (int cc = 0; cc < G_N / 2; cc += 8) {
    const int col = half * (G_N / 2) + cc;
    uint32_t v[8];
    tc_ld8(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)col, v);
    if (i < M) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = j0 + col + q;
        if (j < N) C[(size_t)j * ldc + i] = (all_ok && issued > 0) ? __uint_as_float(v[q]) : 0.0f;
      }
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, G_N);
}

// partial y for the column slice blockIdx.y: part[slice][row]
__global__ void k_gemv_cm(int rows, int cols, int per, const float* __restrict__ W, const float* __restrict__ x,
                          float* __restrict__ part) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = blockIdx.y * per, c1 = min(cols, c0 + per);
  if (r >= rows) return;
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
  int c = c0;
  for (; c + 3 < c1; c += 4) {
    s0 = fmaf(W[(size_t)c * rows + r], __ldg(x + c), s0);
    s1 = fmaf(W[(size_t)(c + 1) * rows + r], __ldg(x + c + 1), s1);
    s2 = fmaf(W[(size_t)(c + 2) * rows + r], __ldg(x + c + 2), s2);
    s3 = fmaf(W[(size_t)(c + 3) * rows + r], __ldg(x + c + 3), s3);
  }
  for (; c < c1; ++c) s0 = fmaf(W[(size_t)c * rows + r], __ldg(x + c), s0);
  part[(size_t)blockIdx.y * rows + r] = (s0 + s1) + (s2 + s3);
}

cudaError_t launch_gemm_tf32x3(bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B,
                               int ldb, float* C, int ldc, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)((M + G_M - 1) / G_M), (unsigned)((N + G_N - 1) / G_N));
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ensure_smem((const void*)kern, G_SMEM);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    kern<<<grid, G_THREADS, G_SMEM, st>>>(M, N, K, A, lda, B, ldb, C, ldc, err);
    return cudaGetLastError();
  };
  if (!ta && !tb) return go(k_gemm_tf32x3<false, false>);
  if (!ta && tb) return go(k_gemm_tf32x3<false, true>);
  if (ta && !tb) return go(k_gemm_tf32x3<true, false>);
  return go(k_gemm_tf32x3<true, true>);
}

int gemv_slices(int cols) { return std::max(1, std::min(32, (cols + 255) / 256)); }

cudaError_t launch_gemv_cm(int rows, int cols, const float* W, const float* x, float* part, cudaStream_t st) {
  const int slices = gemv_slices(cols);
  const int per = (cols + slices - 1) / slices;
  dim3 grid((unsigned)((rows + 127) / 128), (unsigned)slices);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_gemv_cm<<<grid, 128, 0, st>>>(rows, cols, per, W, x, part);
  return cudaGetLastError();
}

}  // namespace lpk
