// lp_adat_noalloc: u = A diag(d2) A^T v for callers that cannot allocate
// device memory.
//
// Who needs this: code that embeds the product in a host application whose
// device memory is fully owned by someone else -- a pre-sized arena, a
// serving loop with a fixed memory budget, or a process where the CUDA
// allocation calls must not be made after start-up (cudaMalloc and cudaFree
// can block or implicitly synchronise the device, and fail once the budget
// is spent).  Such callers cannot use lp_create, which allocates a handle's
// workspaces.  This entry point takes the caller's buffers and keeps its own
// scratch (per-CTA partial vectors, group sums, reduction tickets and a status
// word) in one statically sized __device__ array that lives as long as the
// library is loaded on each device that used it.
//
// Kernel: the same warp-specialised bulk-copy pipeline as the product used
// inside the solver (one producer warp, 16 consumer warps, full/empty
// mbarriers, FP32 products with FP32 per-lane accumulation, a deterministic
// two-level FP64 reduction of the per-CTA partials), except that d2 is read
// in FP64 straight from the caller's vector instead of being staged.
#include <mutex>

#include "../../include/lp_sketch_ipm.h"
#include "internal.h"

namespace lpk {
namespace {

// Scratch layout (bytes): [0, 512) tickets (kMaxGroups + 1 unsigned),
// [512, 528) status word, [1024, ...) group sums (FP64), then per-CTA partials (FP32).
constexpr size_t kNaScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kNaMaxGrid = 160;
constexpr int kNaTicketBytes = 512;
constexpr int kNaStatusOff = 512;
constexpr int kNaGpartOff = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

size_t na_gpart_bytes(int lda) { return (size_t)((kNaMaxGrid + kGroup - 1) / kGroup) * lda * 8; }
size_t na_total_bytes(int lda) {
  return kNaGpartOff + na_gpart_bytes(lda) + (size_t)kNaMaxGrid * lda * 4;
}

struct NaArgs {
  const void* A;
  int lda, m;
  long long n;
  int nb, ntiles, stages;
  const double* d2;
  const double* v;
  double* u;
  float* partials;     // [grid][lda]
  double* gpart;       // [ngroups][lda]
  unsigned* tickets;   // [kMaxGroups + 1]
  int* status;
};

template <typename TA>
__device__ __forceinline__ void na_issue(const NaArgs& a, char* smem, int stage_bytes,
                                         uint64_t* full, int stage, int tile) {
  const long long j0 = (long long)tile * a.nb;
  const int ncols = (int)min((long long)a.nb, a.n - j0);
  const uint32_t bytes = (uint32_t)ncols * (uint32_t)a.lda * (uint32_t)sizeof(TA);
  mbar_arrive_expect_tx(&full[stage], bytes);
  bulk_g2s(smem + (size_t)stage * stage_bytes,
           static_cast<const char*>(a.A) + (size_t)j0 * a.lda * sizeof(TA), bytes, &full[stage]);
}

template <typename TA, int VPL>
__global__ void __launch_bounds__(kFusedThreads, 1) k_adat_noalloc(const NaArgs a) {
  constexpr int VEC = VecOf<TA>::N;
  extern __shared__ __align__(128) char smem[];
  const int stage_bytes = align_up_i(a.nb * a.lda * (int)sizeof(TA), 128);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.stages * stage_bytes);
  uint64_t* empty = full + a.stages;
  float* v_s = reinterpret_cast<float*>(smem + (size_t)a.stages * stage_bytes + 2 * kMaxStages * 8);
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RV = a.lda / VEC;
  const int S = a.stages;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kConsumerWarps);
    }
    fence_mbar_init();
  }
  for (int i = tid; i < a.lda; i += blockDim.x) v_s[i] = (i < a.m) ? (float)a.v[i] : 0.0f;
  __syncthreads();
  float acc[VPL][VEC];
#pragma unroll
  for (int c = 0; c < VPL; ++c)
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[c][e] = 0.0f;
  bool aborted = false;
  if (warp == kConsumerWarps) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < my_tiles; ++i) {
        const int st = i % S;
        if (i >= S && !mbar_wait(&empty[st], (uint32_t)(((i / S) - 1) & 1), a.status)) {
          aborted = true;
          break;
        }
        fence_proxy_async_smem();
        na_issue<TA>(a, smem, stage_bytes, full, st, (int)blockIdx.x + i * (int)gridDim.x);
        issued = i + 1;
      }
      if (aborted || *a.status != ERR_NONE)
        for (int j = (issued > S ? issued - S : 0); j < issued; ++j)
          mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), a.status);
    }
  } else {
    for (int i = 0; i < my_tiles; ++i) {
      const int st = i % S;
      if (!mbar_wait(&full[st], (uint32_t)((i / S) & 1), a.status)) {
        aborted = true;
        break;
      }
      const long long j0 = (long long)((int)blockIdx.x + i * (int)gridDim.x) * a.nb;
      const int ncols = (int)min((long long)a.nb, a.n - j0);
      const TA* At = reinterpret_cast<const TA*>(smem + (size_t)st * stage_bytes);
      for (int jj = warp; jj < ncols; jj += kConsumerWarps) {
        const float d2j = (float)__ldg(a.d2 + j0 + jj);
        const TA* col = At + (size_t)jj * a.lda;
        float av[VPL][VEC];
        float dp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < VPL; ++c) {
          const int rv = c * 32 + lane;
          if (rv < RV) {
            ld16<float>(col + rv * VEC, av[c]);
            // rows m .. ld-1 are the caller's padding and may hold anything
            // (NaN or Inf included): they must not reach the dot product
            if ((rv + 1) * VEC > a.m) {
#pragma unroll
              for (int e = 0; e < VEC; ++e)
                if (rv * VEC + e >= a.m) av[c][e] = 0.0f;
            }
          } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) av[c][e] = 0.0f;
          }
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float vv = (rv < RV) ? v_s[rv * VEC + e] : 0.0f;
            dp[(c * VEC + e) & 3] = fmaf(av[c][e], vv, dp[(c * VEC + e) & 3]);
          }
        }
        const float t = d2j * warp_sum((dp[0] + dp[1]) + (dp[2] + dp[3]));
#pragma unroll
        for (int c = 0; c < VPL; ++c)
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[c][e] = fmaf(av[c][e], t, acc[c][e]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  aborted = __syncthreads_or(aborted) != 0;
  float* buf = reinterpret_cast<float*>(smem);
  if (warp < kConsumerWarps) {
#pragma unroll
    for (int c = 0; c < VPL; ++c) {
      const int rv = c * 32 + lane;
      if (rv < RV)
#pragma unroll
        for (int e = 0; e < VEC; ++e) buf[(size_t)warp * a.lda + rv * VEC + e] = acc[c][e];
    }
  }
  __syncthreads();
  float* part = a.partials + (size_t)blockIdx.x * a.lda;
  for (int r = tid; r < a.lda; r += blockDim.x) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kConsumerWarps; ++w) s += buf[(size_t)w * a.lda + r];
    part[r] = aborted ? 0.0f : s;
  }
  // two-level reduction: group sums, then the last group reducer writes u
  const int G = gridDim.x, ngroups = (G + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup, b0 = grp * kGroup, gsize = min(kGroup, G - b0);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(a.tickets + grp, 1u);
    const bool last = (t == (unsigned)gsize - 1u);
    if (last) a.tickets[grp] = 0u;
    s_flag = last ? 1 : 0;
  }
  __syncthreads();
  if (s_flag == 0) return;
  __threadfence();
  for (int i = tid; i < a.lda; i += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < gsize; ++q) s += (double)__ldcg(a.partials + (size_t)(b0 + q) * a.lda + i);
    a.gpart[(size_t)grp * a.lda + i] = s;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(a.tickets + kMaxGroups, 1u);
    const bool last = (t == (unsigned)ngroups - 1u);
    if (last) a.tickets[kMaxGroups] = 0u;
    s_flag = last ? 1 : 0;
  }
  __syncthreads();
  if (s_flag == 0) return;
  __threadfence();
  for (int i = tid; i < a.m; i += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < ngroups; ++g) s += __ldcg(a.gpart + (size_t)g * a.lda + i);
    a.u[i] = s;
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mutex;
void* g_na_ptr[64] = {nullptr};

template <typename TA, int VPL>
cudaError_t na_launch(const NaArgs& a, int grid, int smem, cudaStream_t st) {
  auto k = k_adat_noalloc<TA, VPL>;
  cudaError_t e = ensure_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k<<<grid, kFusedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename TA>
cudaError_t na_dispatch(int vpl, const NaArgs& a, int grid, int smem, cudaStream_t st) {
  switch (vpl) {
    case 1: return na_launch<TA, 1>(a, grid, smem, st);
    case 2: return na_launch<TA, 2>(a, grid, smem, st);
    case 4: return na_launch<TA, 4>(a, grid, smem, st);
    case 8: return na_launch<TA, 8>(a, grid, smem, st);
    case 16: return na_launch<TA, 16>(a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace lpk

using namespace lpk;

extern "C" int lp_adat_noalloc(const void* A, int32_t dtype, int32_t m, int64_t n, int64_t ld,
                               const double* d2, const double* v, double* u, void* stream) {
  if (!A || !d2 || !v || !u || m < 1 || n < 1 || ld < m) return LP_ERR_ARG;
  if (dtype != LP_F32 && dtype != LP_BF16) return LP_ERR_ARG;
  const int esz = dtype == LP_F32 ? 4 : 2;
  if ((ld * esz) % 16 != 0 || (reinterpret_cast<uintptr_t>(A) % 16) != 0) return LP_ERR_ARG;
  if (ld > (1 << 20)) return LP_ERR_ARG;
  const int lda = (int)ld;
  const int vpl = fused_vpl(lda, esz);
  if (vpl == 0) return LP_ERR_ARG;                              // m beyond the kernel's register tile
  if (na_total_bytes(lda) > kNaScratchBytes) return LP_ERR_ARG;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LP_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LP_ERR_CUDA;
      g_na_ptr[dev] = p;
    }
    base = g_na_ptr[dev];
  }
  int num_sms = 1;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LP_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // tiles of ~32 KB; as many stages as fit next to the v vector and barriers
  const int col_bytes = lda * esz;
  int nb = std::max(4, std::min(64, 32768 / col_bytes)) / 4 * 4;
  const int stage_bytes = align_up_i(nb * col_bytes, 128);
  const int tail = 2 * kMaxStages * 8 + align_up_i(lda * 4, 128) + 128;
  int stages = kMaxStages;
  while (stages > 2 && stages * stage_bytes + tail > 220 * 1024) --stages;
  if (stages * stage_bytes + tail > 227 * 1024) return LP_ERR_ARG;
  if (stages * stage_bytes < kConsumerWarps * lda * 4) return LP_ERR_ARG;
  const long long ntiles = (n + nb - 1) / nb;
  if (ntiles > (1LL << 30)) return LP_ERR_ARG;
  const int grid = (int)std::max(1LL, std::min<long long>(ntiles, std::min(num_sms, kNaMaxGrid)));
  NaArgs a;
  a.A = A;
  a.lda = lda;
  a.m = m;
  a.n = n;
  a.nb = nb;
  a.ntiles = (int)ntiles;
  a.stages = stages;
  a.d2 = d2;
  a.v = v;
  a.u = u;
  unsigned char* b = static_cast<unsigned char*>(base);
  a.tickets = reinterpret_cast<unsigned*>(b);
  a.status = reinterpret_cast<int*>(b + kNaStatusOff);
  a.gpart = reinterpret_cast<double*>(b + kNaGpartOff);
  a.partials = reinterpret_cast<float*>(b + kNaGpartOff + na_gpart_bytes(lda));
  // tickets and the status word must start at zero (a previous call may have aborted)
  if (cudaMemsetAsync(b, 0, kNaGpartOff, st) != cudaSuccess) return LP_ERR_CUDA;
  const int smem = stages * stage_bytes + tail;
  cudaError_t e = dtype == LP_F32 ? na_dispatch<float>(vpl, a, grid, smem, st)
                                  : na_dispatch<bf16raw>(vpl, a, grid, smem, st);
  if (e != cudaSuccess) return LP_ERR_CUDA;
  int status = 0;
  if (cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return LP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LP_ERR_CUDA;
  if (status == ERR_TIMEOUT) return LP_ERR_DEVICE_TIMEOUT;
  return LP_OK;
}
