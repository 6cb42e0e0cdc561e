// Gaussian sketch A D W_G on the 5th-generation tensor cores (tcgen05, TMEM).
//
// C (m x w) = A (m x n) * W' (n x w), with W'_jk = fl32(fl32(d_j) g_jk) drawn
// in the kernel (gauss.cuh).  The contraction runs as tcgen05.mma.kind::tf32
// with FP32 accumulators in tensor memory, and keeps FP32 accuracy by
// splitting each FP32 operand into two TF32 parts, x = x_hi + x_lo with
// x_hi = tf32(x), x_lo = tf32(x - x_hi):
//     A W' ~ A_hi W_hi + A_lo W_hi + A_hi W_lo      (the A_lo W_lo term is below
//                                                   FP32 rounding and dropped)
// BF16 A is exact in TF32 (A_lo = 0), so it takes two products.
//
// Work split: a CTA owns up to MB = 4 row blocks of 128 rows, one 128-column
// block of W' and a slice of the n columns of A (split-K), so for m <= 512
// every W' entry is drawn exactly once.  Per chunk of 16 columns of A, 16
// staging warps stage A_hi, A_lo, W_hi and W_lo in shared memory in the
// K-major core-matrix layout (8 rows x 16 bytes per core matrix, no swizzle)
// and arrive on the chunk's "full" mbarrier; a separate warp waits on it,
// issues the MMAs (M = 128, N = 128, K = 8) and commits them to the chunk's
// "empty" mbarrier, which the stagers wait on before they reuse the buffer.
// Two buffers let the next chunk be staged while the tensor core works, and
// the stagers never wait for the MMA issue itself.  Each row block accumulates in its own 128 TMEM columns.  The
// FP32 tile is added to the FP64 result with atomics.  Every wait is bounded
// and tensor memory is released on every path.
#include "gauss.cuh"

namespace lpk {

namespace {

constexpr int TC_M = 128;       // MMA M: rows of A in one row block
constexpr int TC_N = 128;       // MMA N: columns of W' per CTA
constexpr int TC_BK = 16;       // columns of A per chunk (two MMA k-steps of 8)
constexpr int TC_STAGERS = 512;               // threads that stage A and draw W'
constexpr int TC_THREADS = TC_STAGERS + 32;    // + the warp that issues the MMAs
constexpr int TC_MAXMB = 4;     // row blocks per CTA: MB * 128 TMEM columns <= 512
// K-major, no-swizzle core-matrix layout of a rows x 16 FP32 tile: element
// (r, k) at (r/8)*SBO + (k/4)*LBO + (r%8)*16 + (k%4)*4 bytes.
constexpr int TC_LBO = 128;                  // next core matrix along K
constexpr int TC_SBO = (TC_BK / 4) * 128;    // next group of 8 rows (512 B)
constexpr int TC_BLK = TC_M * TC_BK * 4;     // 8 KB: one 128 x 16 FP32 operand tile
constexpr int TC_SMEM_PER_SM = 228 * 1024;

__host__ __device__ constexpr int stage_bytes(int mb, bool split_a) {
  return (split_a ? 2 : 1) * mb * TC_BLK + 2 * TC_BLK;
}

__host__ __device__ constexpr int tmem_cols(int mb) { return mb == 1 ? 128 : (mb == 2 ? 256 : 512); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // fixed descriptor version of tcgen05
  // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
  return d;
}

// instruction descriptor: kind::tf32, FP32 accumulator, K-major A and B, M = 128, N = 128
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4)      // D format F32
         | (2u << 7)    // A format TF32
         | (2u << 10)   // B format TF32
         | (0u << 15)   // A K-major
         | (0u << 16)   // B K-major
         | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <typename TA>
__device__ __forceinline__ float load_a(const TA* A, size_t idx) {
  if (sizeof(TA) == 4) return reinterpret_cast<const float*>(A)[idx];
  return __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(A)[idx] << 16);
}

__device__ __forceinline__ int core_off(int r, int k4) { return (r >> 3) * TC_SBO + k4 * TC_LBO + (r & 7) * 16; }

}  // namespace

// grid: x = groups of MB row blocks, y = 128-column blocks of W', z = K slices
// named barrier over the staging threads (id 1; 0 is __syncthreads')
__device__ __forceinline__ void stagers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(TC_STAGERS) : "memory");
}

template <typename TA, bool SPLIT_A>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gauss_tc(const TA* __restrict__ A, int lda, int m, long long n, const double* __restrict__ dvec,
               int is_d2, uint64_t s_kr, int w, float inv_sqrt_w, int mb, long long kper,
               double* __restrict__ adw, int* err) {
  extern __shared__ __align__(1024) char smem[];
  __shared__ uint64_t full[2], empty[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ float d_s[2][TC_BK];  // fl32(d_j) of the chunk's columns, double-buffered
  __shared__ int mma_ok_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * mb * TC_M, k0 = blockIdx.y * TC_N;
  const long long j0 = blockIdx.z * kper;
  const long long j1 = min(n, j0 + kper);
  const long long nchunks = j1 > j0 ? (j1 - j0 + TC_BK - 1) / TC_BK : 0;
  const int ncols = tmem_cols(mb);
  const int sbytes = stage_bytes(mb, SPLIT_A);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full[b], TC_STAGERS);
      mbar_init(&empty[b], 1);
    }
    fence_mbar_init();
    mma_ok_s = 1;
  }
  if (tid < TC_BK) d_s[0][tid] = j0 + tid < j1 ? gauss_dval(dvec, j0 + tid, is_d2) : 0.0f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  constexpr uint32_t idesc = make_idesc();
  long long staged = 0;  // chunks this thread staged (stagers) or issued (MMA lane)

  if (warp == TC_STAGERS / 32) {
    // ---------------- the MMA warp: one lane issues, per chunk, the MMAs of
    // the chunk's stage once every staging thread has arrived on full[b], and
    // commits them to empty[b] ----------------
    if (lane == 0) {
      for (long long c = 0; c < nchunks; ++c) {
        const int b = (int)(c & 1);
        if (!mbar_wait(&full[b], (uint32_t)((c >> 1) & 1), err)) {
          mma_ok_s = 0;
          break;
        }
        tc_fence_after();
        const uint32_t s0 = smem_u32(smem + (size_t)b * sbytes);
        const uint32_t whi = s0 + (SPLIT_A ? 2 : 1) * mb * TC_BLK;
        const uint32_t wlo = whi + TC_BLK;
#pragma unroll 1
        for (int rb = 0; rb < mb; ++rb) {
          const uint32_t d = tmem + (uint32_t)(rb * TC_N);
          const uint32_t ahi = s0 + rb * TC_BLK;
          const uint32_t alo = s0 + (mb + rb) * TC_BLK;
#pragma unroll
          for (int s = 0; s < TC_BK / 8; ++s) {
            const uint32_t koff = (uint32_t)(s * 2 * TC_LBO);  // two core matrices per k-step
            tc_mma(d, make_sdesc(ahi + koff), make_sdesc(whi + koff), idesc, (c > 0 || s > 0) ? 1u : 0u);
            tc_mma(d, make_sdesc(ahi + koff), make_sdesc(wlo + koff), idesc, 1u);
            if (SPLIT_A) tc_mma(d, make_sdesc(alo + koff), make_sdesc(whi + koff), idesc, 1u);
          }
        }
        tc_commit(&empty[b]);
        staged = c + 1;
      }
      // no MMA of this CTA may still run when tensor memory is read or freed:
      // the last commit arrives once every MMA issued before it has completed
      if (staged > 0 && !mbar_wait(&empty[(staged - 1) & 1], (uint32_t)(((staged - 1) >> 1) & 1), err))
        mma_ok_s = 0;
    }
  } else {
    // ---------------- the staging threads ----------------
    // thread t owns operand row r = t % 128 and the k4 group g = t / 128
    // (columns 4g .. 4g+3 of the chunk)
    const int r = tid & (TC_M - 1);
    const int g = tid >> 7;
    // A of the next chunk is loaded into registers while the current chunk's W'
    // is drawn, so the global-load latency hides behind the generator
    float an[TC_MAXMB][4];
    auto load_chunk = [&](long long jb) {
#pragma unroll
      for (int rb = 0; rb < TC_MAXMB; ++rb) {
        const int i = i0 + rb * TC_M + r;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const long long j = jb + g * 4 + q;
          an[rb][q] = (rb < mb && i < m && j < j1) ? load_a<TA>(A, (size_t)j * lda + i) : 0.0f;
        }
      }
    };
    if (nchunks > 0) load_chunk(j0);
    bool ok = true;
    for (long long c = 0; c < nchunks; ++c) {
      const int b = (int)(c & 1);
      char* stage = smem + (size_t)b * sbytes;
      // the MMAs that last read this buffer (chunk c - 2) must have completed
      if (c >= 2 && ok) ok = mbar_wait(&empty[b], (uint32_t)(((c - 2) >> 1) & 1), err);
      ok = ok && *reinterpret_cast<volatile int*>(&mma_ok_s) != 0;
      const long long jb = j0 + c * TC_BK;
      // d of the next chunk into the other buffer; its last readers (chunk c - 1)
      // passed the staging barrier that ended chunk c - 1
      if (tid < TC_BK) {
        const long long jn = jb + TC_BK + tid;
        d_s[(c + 1) & 1][tid] = jn < j1 ? gauss_dval(dvec, jn, is_d2) : 0.0f;
      }
      if (ok) {
        // ---- A: MB row blocks, split into TF32 hi / lo ----
#pragma unroll
        for (int rb = 0; rb < TC_MAXMB; ++rb) {
          if (rb < mb) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              hi[q] = to_tf32(an[rb][q]);
              lo[q] = SPLIT_A ? to_tf32(an[rb][q] - __uint_as_float(hi[q])) : 0u;
            }
            const int off = rb * TC_BLK + core_off(r, g);
            *reinterpret_cast<uint4*>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            if (SPLIT_A)
              *reinterpret_cast<uint4*>(stage + mb * TC_BLK + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      }
      if (c + 1 < nchunks) load_chunk(jb + TC_BK);
      if (ok) {
        // ---- W': operand rows are the columns k of W', K runs over j.  With w
        // even, entries (j, k) and (j, k + 1) for even k are the two normals of
        // one Box-Muller draw (counter (j w + k) / 2), so thread t draws both for
        // the column pair k0 + 2 (t % 64) and the rows jb + 2 (t / 64) + {0, 1};
        // for odd w every entry is drawn on its own ----
        char* whi = stage + (SPLIT_A ? 2 : 1) * mb * TC_BLK;
        char* wlo = whi + TC_BLK;
        const int kr = 2 * (tid & 63);        // operand rows kr, kr + 1
        const int jc = 2 * (tid >> 6);        // K columns jc, jc + 1 of the chunk
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
          const long long j = jb + jc + dj;
          const float djv = d_s[c & 1][jc + dj];
          float gv[2] = {0.0f, 0.0f};
          if (j < j1 && k0 + kr < w) {
            if ((w & 1) == 0) {
              gauss_pair(s_kr, ((uint64_t)j * w + (uint64_t)(k0 + kr)) >> 1, inv_sqrt_w, &gv[0], &gv[1]);
              if (k0 + kr + 1 >= w) gv[1] = 0.0f;
            } else {
              gv[0] = gauss_entry(s_kr, (uint64_t)j * w + (uint64_t)(k0 + kr), inv_sqrt_w);
              if (k0 + kr + 1 < w) gv[1] = gauss_entry(s_kr, (uint64_t)j * w + (uint64_t)(k0 + kr + 1), inv_sqrt_w);
            }
          }
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float wv = __fmul_rn(djv, gv[e]);
            const uint32_t hi = to_tf32(wv);
            const uint32_t lo = to_tf32(wv - __uint_as_float(hi));
            const int row = kr + e, col = jc + dj;
            const int off = (row >> 3) * TC_SBO + (col >> 2) * TC_LBO + (row & 7) * 16 + (col & 3) * 4;
            *reinterpret_cast<uint32_t*>(whi + off) = hi;
            *reinterpret_cast<uint32_t*>(wlo + off) = lo;
          }
        }
      }
      // make the generic-proxy stores visible to the tensor core, then hand the
      // stage to the MMA lane; the staging barrier also keeps the threads one
      // chunk apart at most (d_s is double-buffered)
      fence_proxy_async_smem();
      mbar_arrive(&full[b]);
      stagers_sync();
      staged = c + 1;
    }
    // wait for the last commits: the last one covers every MMA issued before
    // it, and waiting on the other buffer's last one leaves no arrive pending
    for (long long c = (staged > 2 ? staged - 2 : 0); c < staged && ok; ++c)
      ok = mbar_wait(&empty[c & 1], (uint32_t)((c >> 1) & 1), err);
    staged = ok ? staged : -1;
  }
  // every thread's outcome: the stagers' waits and the MMA lane's
  const bool all_ok = __syncthreads_and(staged >= 0 && mma_ok_s != 0) != 0;
  tc_fence_after();
  if (all_ok && nchunks > 0 && warp < TC_STAGERS / 32) {
    // warp q reads TMEM lanes [32 (q % 4), +32) and quarter q / 4 of the columns
    const int lg = warp & 3, quarter = warp >> 2;
    for (int rb = 0; rb < mb; ++rb) {
      const int i = i0 + rb * TC_M + lg * 32 + lane;
#pragma unroll 1
      for (int cc = 0; cc < TC_N / 4; cc += 8) {
        const int col = quarter * (TC_N / 4) + cc;
        uint32_t v[8];
        const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(rb * TC_N + col);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (i < m) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int k = k0 + col + q;
            if (k < w) atomicAdd(&adw[(size_t)i * w + k], (double)__uint_as_float(v[q]));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

cudaError_t launch_gauss_tc(int dtype, const void* A, int lda, int m, long long n, const double* dvec,
                            int is_d2, uint64_t s_kr, int w, float inv_sqrt_w, double* adw, int* err,
                            int num_sms, cudaStream_t st) {
  if (dtype != 1 && dtype != 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(adw, 0, sizeof(double) * (size_t)m * w, st);
  if (e != cudaSuccess || n <= 0 || m <= 0 || w <= 0) return e;
  const int gx = (m + TC_M - 1) / TC_M;
  const int mb = std::min(TC_MAXMB, gx);
  const int gxb = (gx + mb - 1) / mb, gy = (w + TC_N - 1) / TC_N;
  // one CTA per SM: K slices so that the grid fills the SMs once
  long long ks = std::max<long long>(1, num_sms / (long long)(gxb * gy));
  ks = std::min<long long>(ks, (n + TC_BK - 1) / TC_BK);
  const long long kper = ((n + ks - 1) / ks + TC_BK - 1) / TC_BK * TC_BK;
  ks = (n + kper - 1) / kper;
  const bool split = dtype == 1;
  // at most 512 / tmem_cols(mb) CTAs may share an SM, so tcgen05.alloc never waits
  const int max_ctas = 512 / tmem_cols(mb);
  const int smem = std::max(2 * stage_bytes(mb, split), TC_SMEM_PER_SM / (max_ctas + 1) + 1024);
  dim3 grid((unsigned)gxb, (unsigned)gy, (unsigned)ks);
  if (split) {
    e = ensure_smem((const void*)k_gauss_tc<float, true>, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_gauss_tc<float, true><<<grid, TC_THREADS, smem, st>>>(static_cast<const float*>(A), lda, m, n, dvec,
                                                           is_d2, s_kr, w, inv_sqrt_w, mb, kper, adw, err);
  } else {
    e = ensure_smem((const void*)k_gauss_tc<bf16raw, false>, smem);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_gauss_tc<bf16raw, false><<<grid, TC_THREADS, smem, st>>>(static_cast<const bf16raw*>(A), lda, m, n,
                                                              dvec, is_d2, s_kr, w, inv_sqrt_w, mb, kper,
                                                              adw, err);
  }
  return cudaGetLastError();
}

}  // namespace lpk
