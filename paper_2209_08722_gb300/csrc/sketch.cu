// CountSketch A D W (Section 2, eq. pdprec; Algorithm 1 step 1) and the
// gather of the correction vector v (eq. compv).
//
// W (n x w) has s nonzeros per row: block b of width wb = w/s holds entry
// sign_b(j)/sqrt(s) at column b*wb + h_b(j), with (h_b(j), sign_b(j)) from the
// SplitMix64 counter-based generator (common.cuh).  W is never stored.
//
// Column g of A D W is the signed, scaled sum of the columns j of A hashed to
// bucket g.  The sketch is built in four passes:
//   1. k_cs_count: bucket sizes (shared-memory histograms) and the per-column
//      scale d_j / sqrt(s), in FP64 and as a double-float pair;
//   2. k_cs_scan: bucket offsets (exclusive scan);
//   3. k_cs_scatter: the bucket lists, entry = j | sign << 31;
//   4. k_cs_bucket: one CTA per bucket sorts its bucket's list by j in shared
//      memory; one producer lane streams the listed columns, whole, with
//      cp.async.bulk into a ring of shared-memory stages, and 512 consumer
//      threads, each owning a few consecutive rows, add every staged column
//      into double-float accumulators in registers (FP64 for FP64 storage).
//      Columns of at most 512 or of more than 4096 rows (or more than the
//      ring holds) take k_cs_accum: one CTA per (bucket, 512-row slab) whose
//      8 warps load their share of the columns themselves and combine partial
//      sums in warp order.
// A is read s times in total (once per listed column).  FP32/BF16 storage
// sums in double-float arithmetic (products formed exactly, relative error
// ~2^-44); FP64 storage sums in FP64.  The summation order depends only on the
// hashes, so the result is bitwise reproducible (for buckets of at most
// kSortCap columns; larger buckets are summed in list order).
#include "internal.h"
#include "df.cuh"

#include <type_traits>

namespace lpk {

namespace {
constexpr int kAccThreads = 256;
constexpr int kAccWarps = kAccThreads / 32;
constexpr int kEPL = 16;                // accumulated elements per lane
constexpr int kSlab = 32 * kEPL;        // rows per CTA
constexpr int kSortCap = 8192;          // bucket entries sorted in shared memory
}  // namespace

// bucket sizes + per-column scales; grid-stride over columns, histogram in smem
__global__ void __launch_bounds__(256) k_cs_count(long long n, int s_blocks, int wb, int w, uint64_t seed,
                                                  long long k, int retry, const double* __restrict__ dvec,
                                                  int is_d2, double inv_sqrt_s, int* __restrict__ count,
                                                  double* __restrict__ sc64, float2* __restrict__ scdf) {
  extern __shared__ int hs[];  // [w]
  for (int g = threadIdx.x; g < w; g += blockDim.x) hs[g] = 0;
  __syncthreads();
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    for (int b = 0; b < s_blocks; ++b) {
      int col;
      float sg;
      cs_entry(seed, k, retry, b, j, wb, &col, &sg);
      atomicAdd(&hs[col], 1);
    }
    const double d = dvec[j];
    const double sc = (is_d2 ? sqrt(d) : d) * inv_sqrt_s;
    sc64[j] = sc;
    const float hi = (float)sc;
    scdf[j] = make_float2(hi, (float)(sc - (double)hi));
  }
  __syncthreads();
  for (int g = threadIdx.x; g < w; g += blockDim.x)
    if (hs[g]) atomicAdd(&count[g], hs[g]);
}

// base[g] = sum of count[0..g), base[w] = total; cursor = base (one CTA)
__global__ void __launch_bounds__(1024) k_cs_scan(int w, const int* __restrict__ count, int* __restrict__ base,
                                                  int* __restrict__ cursor) {
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (w + blockDim.x - 1) / blockDim.x;
  const int g0 = min(w, tid * per), g1 = min(w, g0 + per);
  int local = 0;
  for (int g = g0; g < g1; ++g) local += count[g];
  // exclusive scan of the per-thread sums
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    wsum[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  int run = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
  for (int g = g0; g < g1; ++g) {
    base[g] = run;
    cursor[g] = run;
    run += count[g];
  }
  if (tid == blockDim.x - 1) base[w] = run;
}

// bucket lists: entry = j | (sign < 0) << 31, in arbitrary order within a bucket
__global__ void __launch_bounds__(256) k_cs_scatter(long long n, int s_blocks, int wb, uint64_t seed, long long k,
                                                    int retry, int* __restrict__ cursor, int* __restrict__ list) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    for (int b = 0; b < s_blocks; ++b) {
      int col;
      float sg;
      cs_entry(seed, k, retry, b, j, wb, &col, &sg);
      const int pos = atomicAdd(&cursor[col], 1);
      list[pos] = (int)j | (sg < 0.0f ? (int)0x80000000u : 0);
    }
  }
}

template <typename TA>
struct AccOf {  // double-float accumulators for FP32/BF16 storage, FP64 for FP64
  static constexpr bool kDF = sizeof(TA) != 8;
};

// one CTA per (bucket g, slab of 512 rows)
template <typename TA>
__global__ void __launch_bounds__(kAccThreads, 2) k_cs_accum(const TA* __restrict__ A, int lda, int m, int w,
                                                          const int* __restrict__ base,
                                                          const int* __restrict__ list,
                                                          const double* __restrict__ sc64,
                                                          const float2* __restrict__ scdf,
                                                          double* __restrict__ adw) {
  constexpr int VEC = VecOf<TA>::N;
  constexpr int NV = kEPL / VEC;  // 16-byte vectors per lane per column
  constexpr bool DF = AccOf<TA>::kDF;
  extern __shared__ __align__(16) char smem[];
  int* keys = reinterpret_cast<int*>(smem);                                  // [kSortCap]
  char* comb = smem + kSortCap * sizeof(int);                                // [warps][kSlab] partials
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = blockIdx.x;
  const int r0 = blockIdx.y * kSlab;
  const int beg = base[g];
  const int cnt = base[g + 1] - beg;

  // ---- the bucket's list, sorted by column index (bitonic sort in smem) ----
  const int* lst = list + beg;
  if (cnt <= kSortCap) {
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    for (int e = tid; e < p2; e += kAccThreads) keys[e] = e < cnt ? lst[e] : 0x7FFFFFFF;
    __syncthreads();
    for (int size = 2; size <= p2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int e = tid; e < (p2 >> 1); e += kAccThreads) {
          const int lo = 2 * e - (e & (stride - 1));
          const int hi = lo + stride;
          const bool up = (lo & size) == 0;
          const int a = keys[lo], b = keys[hi];
          const bool gt = (a & 0x7FFFFFFF) > (b & 0x7FFFFFFF);
          if (gt == up) {
            keys[lo] = b;
            keys[hi] = a;
          }
        }
        __syncthreads();
      }
    }
    lst = keys;
  }

  // ---- warp p sums entries [cnt p / 8, cnt (p + 1) / 8) ----
  const int e0 = (int)((long long)cnt * warp / kAccWarps);
  const int e1 = (int)((long long)cnt * (warp + 1) / kAccWarps);
  float hi[kEPL], lo[kEPL];
  double acc[DF ? 1 : kEPL];
#pragma unroll
  for (int q = 0; q < kEPL; ++q) {
    hi[q] = 0.0f;
    lo[q] = 0.0f;
  }
#pragma unroll
  for (int q = 0; q < (DF ? 1 : kEPL); ++q) acc[q] = 0.0;

  // loaded elements: FP32 for FP32/BF16 storage (exact), FP64 for FP64; a ring
  // of D columns per lane keeps D - 1 to D column loads in flight per warp
  using LT = typename std::conditional<DF, float, double>::type;
  constexpr int D = DF ? 3 : 2;
  LT buf[D][kEPL];
  int key[D];
  auto load = [&](int e, LT (&v)[kEPL], int& kk) {
    kk = lst[e];
    const long long j = kk & 0x7FFFFFFF;
    const TA* col = A + (size_t)j * lda + r0;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int row = t * 32 * VEC + lane * VEC;
      if (r0 + row < lda) {
        ld16<LT>(col + row, &v[t * VEC]);
      } else {
#pragma unroll
        for (int q = 0; q < VEC; ++q) v[t * VEC + q] = (LT)0;
      }
    }
  };
#pragma unroll
  for (int u = 0; u < D; ++u)
    if (e0 + u < e1) load(e0 + u, buf[u], key[u]);
  for (int eb = e0; eb < e1; eb += D) {
#pragma unroll
    for (int u = 0; u < D; ++u) {
      const int e = eb + u;
      if (e >= e1) break;
      const long long j = key[u] & 0x7FFFFFFF;
      const bool neg = key[u] < 0;
      if (DF) {
        const float2 sc = scdf[j];
        const float sh = neg ? -sc.x : sc.x, sl = neg ? -sc.y : sc.y;
#pragma unroll
        for (int q = 0; q < kEPL; ++q) df_fma((float)buf[u][q], sh, sl, hi[q], lo[q]);
        // keep |lo| near ulp(hi): its own rounding then stays ~2^-48 |hi| per step
        if (((e - e0) & 7) == 7) {
#pragma unroll
          for (int q = 0; q < kEPL; ++q) df_renorm(hi[q], lo[q]);
        }
      } else {
        const double sc = neg ? -sc64[j] : sc64[j];
#pragma unroll
        for (int q = 0; q < (DF ? 1 : kEPL); ++q) acc[q] = fma((double)buf[u][q], sc, acc[q]);
      }
      if (e + D < e1) load(e + D, buf[u], key[u]);
    }
  }

  // ---- combine the warps' partial sums in warp order ----
  __syncthreads();  // the sorted keys are no longer read; comb may be written
#pragma unroll
  for (int t = 0; t < NV; ++t)
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      const int row = t * 32 * VEC + lane * VEC + q;
      if (DF)
        reinterpret_cast<float2*>(comb)[warp * kSlab + row] = make_float2(hi[t * VEC + q], lo[t * VEC + q]);
      else
        reinterpret_cast<double*>(comb)[warp * kSlab + row] = acc[DF ? 0 : t * VEC + q];
    }
  __syncthreads();
  for (int row = tid; row < kSlab; row += kAccThreads) {
    const int i = r0 + row;
    if (i >= m) continue;
    double out;
    if (DF) {
      const float2* cp = reinterpret_cast<const float2*>(comb);
      float sh = cp[row].x, sl = cp[row].y;
      for (int p = 1; p < kAccWarps; ++p) df_add(sh, sl, cp[p * kSlab + row].x, cp[p * kSlab + row].y);
      out = (double)sh + (double)sl;
    } else {
      const double* cp = reinterpret_cast<const double*>(comb);
      out = cp[row];
      for (int p = 1; p < kAccWarps; ++p) out += cp[p * kSlab + row];
    }
    adw[(size_t)i * w + g] = out;
  }
}

namespace {
constexpr int kBkConsumers = 16;                      // consumer warps of k_cs_bucket
constexpr int kBkThreads = (kBkConsumers + 1) * 32;   // + one producer warp
constexpr int kBkRows = kBkConsumers * 32;            // threads that own rows
constexpr int kBkRingBytes = 48 * 1024;               // column ring per CTA
constexpr int kBkMaxStages = 32;
constexpr int kBkSortCap = 4096;                      // bucket entries sorted (and scaled) in smem

// RPT consecutive elements of a staged column, converted to FP32 (FP32/BF16
// storage) or FP64
template <typename TA, int RPT, typename LT>
__device__ __forceinline__ void bk_load(const TA* p, LT (&v)[RPT]) {
  if constexpr (sizeof(TA) == 2) {
    static_assert(RPT % 2 == 0, "BF16 rows come in pairs");
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int r = 0; r < RPT / 2; ++r) {
      const uint32_t x = q[r];
      v[2 * r] = (LT)__uint_as_float(x << 16);
      v[2 * r + 1] = (LT)__uint_as_float(x & 0xFFFF0000u);
    }
  } else {
#pragma unroll
    for (int r = 0; r < RPT; ++r) v[r] = (LT)p[r];
  }
}
}  // namespace

// One CTA per bucket g, all rows: the bucket's list is sorted by column index
// in shared memory and the signed scale of every listed column gathered next
// to it; then one producer lane streams the listed columns (whole, lda
// elements, contiguous in the column-major A) with cp.async.bulk into a ring
// of shared-memory stages, and each of the 512 consumer threads adds its RPT
// consecutive rows of every staged column, in list order, into double-float
// accumulators in registers (FP64 for FP64 storage).  A is read once per
// listed column, with up to `stages` columns in flight per CTA; the sum of
// every output element runs over the bucket's columns in increasing j, so the
// result is bitwise reproducible (buckets of at most kBkSortCap columns;
// larger ones are summed in list order, their scales read from global
// memory).  Waits are bounded; on a timeout the producer waits (bounded) for
// its copies in flight and the bucket's column is written as zeros.
template <typename TA, int RPT>
__global__ void __launch_bounds__(kBkThreads, 2) k_cs_bucket(const TA* __restrict__ A, int lda, int m, int w,
                                                             int stages, const int* __restrict__ base,
                                                             const int* __restrict__ list,
                                                             const double* __restrict__ sc64,
                                                             const float2* __restrict__ scdf,
                                                             double* __restrict__ adw, int* err) {
  constexpr bool DF = sizeof(TA) != 8;
  using LT = typename std::conditional<DF, float, double>::type;
  extern __shared__ __align__(16) char smem[];
  const int col_bytes = lda * (int)sizeof(TA);
  char* ring = smem;                                                          // [stages][col_bytes]
  int* keys = reinterpret_cast<int*>(smem + (size_t)stages * col_bytes);     // [kBkSortCap]
  uint64_t* scs = reinterpret_cast<uint64_t*>(keys + kBkSortCap);           // [kBkSortCap] signed scales
  uint64_t* full = scs + kBkSortCap;                                         // [stages]
  uint64_t* empty = full + stages;                                           // [stages]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = blockIdx.x;
  const int beg = base[g];
  const int cnt = base[g + 1] - beg;

  if (tid == 0) {
    for (int st = 0; st < stages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kBkConsumers);
    }
    fence_mbar_init();
  }
  // ---- the bucket's list, sorted by column index (bitonic sort in smem) ----
  const int* lst = list + beg;
  const bool sorted = cnt <= kBkSortCap;
  if (sorted) {
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    for (int e = tid; e < p2; e += kBkThreads) keys[e] = e < cnt ? lst[e] : 0x7FFFFFFF;
    __syncthreads();
    for (int size = 2; size <= p2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int e = tid; e < (p2 >> 1); e += kBkThreads) {
          const int lo = 2 * e - (e & (stride - 1));
          const int hi = lo + stride;
          const bool up = (lo & size) == 0;
          const int a = keys[lo], b = keys[hi];
          const bool gt = (a & 0x7FFFFFFF) > (b & 0x7FFFFFFF);
          if (gt == up) {
            keys[lo] = b;
            keys[hi] = a;
          }
        }
        __syncthreads();
      }
    }
    lst = keys;
    // the signed scale of every listed column, gathered once (the loads of all
    // entries in flight together) instead of once per column in the loop
    for (int e = tid; e < cnt; e += kBkThreads) {
      const int key = keys[e];
      const long long j = key & 0x7FFFFFFF;
      if constexpr (DF) {
        float2 sc = scdf[j];
        if (key < 0) sc = make_float2(-sc.x, -sc.y);
        scs[e] = ((uint64_t)__float_as_uint(sc.y) << 32) | __float_as_uint(sc.x);
      } else {
        const double sc = key < 0 ? -sc64[j] : sc64[j];
        scs[e] = (uint64_t)__double_as_longlong(sc);
      }
    }
  }
  __syncthreads();  // barriers initialised, keys sorted, scales gathered

  if (warp == kBkConsumers) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int st = 0, issued = 0;
      uint32_t parity = 1u;  // phase of empty[st] to wait for (the first pass waits for none)
      bool aborted = false;
      for (int e = 0; e < cnt; ++e) {
        if (e >= stages && !mbar_wait(&empty[st], parity, err)) {
          aborted = true;
          break;
        }
        fence_proxy_async_smem();
        const long long j = lst[e] & 0x7FFFFFFF;
        mbar_arrive_expect_tx(&full[st], (uint32_t)col_bytes);
        bulk_g2s(ring + (size_t)st * col_bytes, A + (size_t)j * lda, (uint32_t)col_bytes, &full[st]);
        issued = e + 1;
        if (++st == stages) {
          st = 0;
          parity ^= 1u;
        }
      }
      if (aborted || *err != ERR_NONE)
        for (int e = (issued > stages ? issued - stages : 0); e < issued; ++e)
          mbar_wait(&full[e % stages], (uint32_t)((e / stages) & 1), err);
    }
    return;
  }
  // ---------------- consumers: rows r0 .. r0 + RPT - 1 ----------------
  const int r0 = tid * RPT;
  const bool rows_ok = r0 < lda;
  float hi[RPT], lo[RPT];
  double acc[DF ? 1 : RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) hi[r] = lo[r] = 0.0f;
#pragma unroll
  for (int r = 0; r < (DF ? 1 : RPT); ++r) acc[r] = 0.0;
  // columns are taken in pairs (stages is even, so a pair's two stages share
  // their phase): one wait and one release per stage as before, but half the
  // loop overhead per column and two independent columns in flight per row
  bool ok = true;
  int st = 0;
  uint32_t parity = 0;
  auto scale_of = [&](int e) -> uint64_t {
    if (sorted) return scs[e];
    const int key = lst[e];
    const long long j = key & 0x7FFFFFFF;
    if constexpr (DF) {
      float2 sc = scdf[j];
      if (key < 0) sc = make_float2(-sc.x, -sc.y);
      return ((uint64_t)__float_as_uint(sc.y) << 32) | __float_as_uint(sc.x);
    } else {
      return (uint64_t)__double_as_longlong(key < 0 ? -sc64[j] : sc64[j]);
    }
  };
  for (int e = 0; e < cnt; e += 2) {
    const bool two = e + 1 < cnt;
    ok = mbar_wait(&full[st], parity, err);
    if (ok && two) ok = mbar_wait(&full[st + 1], parity, err);
    if (!ok) break;
    if (rows_ok) {
      LT v0[RPT], v1[RPT];
      const uint64_t b0 = scale_of(e);
      const uint64_t b1 = two ? scale_of(e + 1) : 0ull;
      bk_load<TA, RPT, LT>(reinterpret_cast<const TA*>(ring + (size_t)st * col_bytes) + r0, v0);
      if (two) bk_load<TA, RPT, LT>(reinterpret_cast<const TA*>(ring + (size_t)(st + 1) * col_bytes) + r0, v1);
      if constexpr (DF) {
        const float h0 = __uint_as_float((uint32_t)b0), l0 = __uint_as_float((uint32_t)(b0 >> 32));
        const float h1 = __uint_as_float((uint32_t)b1), l1 = __uint_as_float((uint32_t)(b1 >> 32));
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          df_fma(v0[r], h0, l0, hi[r], lo[r]);
          if (two) df_fma(v1[r], h1, l1, hi[r], lo[r]);
        }
        if ((e & 7) == 6) {  // after column e + 1 = 7 (mod 8)
#pragma unroll
          for (int r = 0; r < RPT; ++r) df_renorm(hi[r], lo[r]);
        }
      } else {
        const double c0 = __longlong_as_double((long long)b0), c1 = __longlong_as_double((long long)b1);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          acc[(DF ? 0 : r)] = fma((double)v0[r], c0, acc[(DF ? 0 : r)]);
          if (two) acc[(DF ? 0 : r)] = fma((double)v1[r], c1, acc[(DF ? 0 : r)]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[st]);
      if (two) mbar_arrive(&empty[st + 1]);
    }
    st += 2;
    if (st == stages) {
      st = 0;
      parity ^= 1u;
    }
  }
  if (!rows_ok) return;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = r0 + r;
    if (i >= m) break;
    double out = DF ? (double)hi[r] + (double)lo[r] : acc[DF ? 0 : r];
    adw[(size_t)i * w + g] = ok ? out : 0.0;
  }
}

// v_i = sqrt(x_i s_i) / sqrt(s) * sum_b sign_b(i) u[col_b(i)]   (eq. compv with u = (ADW)^+ r)
__global__ void k_v_gather(long long n, const double* __restrict__ x, const double* __restrict__ s,
                           const double* __restrict__ u, uint64_t seed, long long k, int retry,
                           int s_blocks, int wb, double scale, double* __restrict__ v) {
  const double inv_sqrt_s = scale / sqrt((double)s_blocks);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < s_blocks; ++b) {
      int col;
      float sg;
      cs_entry(seed, k, retry, b, i, wb, &col, &sg);
      acc += (double)sg * u[col];
    }
    const double xs = s ? x[i] * s[i] : x[i];  // s == nullptr: x holds x o s
    v[i] = sqrt(xs) * inv_sqrt_s * acc;
  }
}

// the bucket sizes, offsets and lists and the per-column scales (passes 1-3)
static cudaError_t cs_lists(long long n, const double* dvec, int is_d2, uint64_t seed, long long k, int retry,
                            int s_blocks, int w, const CsWork& ws, int num_sms, cudaStream_t st) {
  const int wb = w / s_blocks;
  const double inv_sqrt_s = 1.0 / sqrt((double)s_blocks);
  cudaError_t e = cudaMemsetAsync(ws.count, 0, sizeof(int) * (size_t)w, st);
  if (e != cudaSuccess) return e;
  const int hist_smem = w * (int)sizeof(int);
  e = ensure_smem((const void*)k_cs_count, hist_smem);
  if (e != cudaSuccess) return e;
  const int grid_cols = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 2));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_cs_count<<<grid_cols, 256, hist_smem, st>>>(n, s_blocks, wb, w, seed, k, retry, dvec, is_d2, inv_sqrt_s,
                                                ws.count, ws.sc64, ws.scdf);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_cs_scan<<<1, 1024, 0, st>>>(w, ws.count, ws.base, ws.cursor);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_cs_scatter<<<grid_cols, 256, 0, st>>>(n, s_blocks, wb, seed, k, retry, ws.cursor, ws.list);
  return cudaGetLastError();
}

// One CTA per bucket g of the sketch of a CSC A: the bucket's column list is
// sorted by j; the entries of the listed columns are gathered into shared
// memory in that order (value times the column's signed scale, in FP64) and
// sorted by (row, gather position); each row's run is then summed in that
// order by one thread and written to ADW (every row of the bucket's column
// that no entry reaches keeps the zero the caller wrote).  So the sum of every
// element runs over its terms in increasing j, whatever the scheduling: the
// result is bitwise reproducible.  A bucket with more than kSpCap entries (or
// a longer list than kBkSortCap) is summed with FP64 atomics instead.
namespace {
constexpr int kSpThreads = 256;
constexpr int kSpCap = 4096;       // gathered entries per bucket
constexpr int kSpPosBits = 12;     // gather position bits of a sort key (kSpCap = 2^12)
}  // namespace

template <typename TV>
__global__ void __launch_bounds__(kSpThreads) k_sp_bucket(const long long* __restrict__ cp, const int* __restrict__ ri,
                                                          const TV* __restrict__ val, int w,
                                                          const int* __restrict__ base, const int* __restrict__ list,
                                                          const double* __restrict__ sc64, double* __restrict__ adw) {
  extern __shared__ __align__(16) char smem[];
  int* keys = reinterpret_cast<int*>(smem);                         // [kBkSortCap] the sorted list
  int* offs = keys + kBkSortCap;                                     // [kBkSortCap + 1] gather offsets
  uint32_t* ek = reinterpret_cast<uint32_t*>(offs + kBkSortCap + 1); // [kSpCap] (row, position) keys
  double* ev = reinterpret_cast<double*>(smem + (size_t)(2 * kBkSortCap + 1 + kSpCap) * 4 + 4);  // [kSpCap]
  __shared__ int s_total;
  const int tid = threadIdx.x;
  const int g = blockIdx.x;
  const int beg = base[g];
  const int cnt = base[g + 1] - beg;
  const int* lst = list + beg;
  if (cnt > kBkSortCap) {  // (very large buckets) FP64 atomics
    for (int e = tid; e < cnt; e += kSpThreads) {
      const int key = lst[e];
      const long long j = key & 0x7FFFFFFF;
      const double sc = key < 0 ? -sc64[j] : sc64[j];
      for (long long q = cp[j]; q < cp[j + 1]; ++q) atomicAdd(&adw[(size_t)ri[q] * w + g], (double)val[q] * sc);
    }
    return;
  }
  // ---- the list, sorted by j ----
  int p2 = 1;
  while (p2 < cnt) p2 <<= 1;
  for (int e = tid; e < p2; e += kSpThreads) keys[e] = e < cnt ? lst[e] : 0x7FFFFFFF;
  __syncthreads();
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = tid; e < (p2 >> 1); e += kSpThreads) {
        const int lo = 2 * e - (e & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const int a = keys[lo], b = keys[hi];
        const bool gt = (a & 0x7FFFFFFF) > (b & 0x7FFFFFFF);
        if (gt == up) {
          keys[lo] = b;
          keys[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  // ---- gather offsets: exclusive scan of the listed columns' entry counts
  // (loaded in parallel; each thread scans a contiguous chunk, one thread the
  // chunk totals) ----
  __shared__ int chunk[kSpThreads];
  for (int e = tid; e < cnt; e += kSpThreads) {
    const long long j = keys[e] & 0x7FFFFFFF;
    const long long len = cp[j + 1] - cp[j];
    offs[e] = (int)std::min<long long>(len, kSpCap + 1);  // larger counts only need to exceed the cap
  }
  __syncthreads();
  const int per = (cnt + kSpThreads - 1) / kSpThreads;
  const int c0 = tid * per, c1 = std::min(cnt, c0 + per);
  int run = 0;
  for (int e = c0; e < c1; ++e) run += offs[e];
  chunk[tid] = run;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < kSpThreads; ++t) {
      const int v = chunk[t];
      chunk[t] = acc;
      acc = std::min(acc + v, kSpCap + 1);
    }
    s_total = acc;
  }
  __syncthreads();
  run = chunk[tid];
  for (int e = c0; e < c1; ++e) {
    const int v = offs[e];
    offs[e] = run;
    run += v;
  }
  if (tid == 0) offs[cnt] = s_total;
  __syncthreads();
  const int total = s_total;
  if (total > kSpCap) {  // too many entries to sort here: FP64 atomics
    for (int e = tid; e < cnt; e += kSpThreads) {
      const int key = keys[e];
      const long long j = key & 0x7FFFFFFF;
      const double sc = key < 0 ? -sc64[j] : sc64[j];
      for (long long q = cp[j]; q < cp[j + 1]; ++q) atomicAdd(&adw[(size_t)ri[q] * w + g], (double)val[q] * sc);
    }
    return;
  }
  // ---- gather: entry q of listed column e at position offs[e] + (q - cp[j]) ----
  for (int e = tid; e < cnt; e += kSpThreads) {
    const int key = keys[e];
    const long long j = key & 0x7FFFFFFF;
    const double sc = key < 0 ? -sc64[j] : sc64[j];
    const long long q0 = cp[j];
    const int o = offs[e], len = offs[e + 1] - o;
#pragma unroll 4
    for (int t = 0; t < len; ++t) {
      ek[o + t] = ((uint32_t)ri[q0 + t] << kSpPosBits) | (uint32_t)(o + t);
      ev[o + t] = (double)val[q0 + t] * sc;
    }
  }
  int t2 = 1;
  while (t2 < total) t2 <<= 1;
  for (int e = total + tid; e < t2; e += kSpThreads) ek[e] = 0xFFFFFFFFu;
  __syncthreads();
  // ---- sort by (row, gather position) ----
  for (int size = 2; size <= t2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = tid; e < (t2 >> 1); e += kSpThreads) {
        const int lo = 2 * e - (e & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint32_t a = ek[lo], b = ek[hi];
        if ((a > b) == up) {
          ek[lo] = b;
          ek[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  // ---- each row's run summed in gather order by the thread at its start ----
  for (int i = tid; i < total; i += kSpThreads) {
    const uint32_t row = ek[i] >> kSpPosBits;
    if (i > 0 && (ek[i - 1] >> kSpPosBits) == row) continue;
    double sum = 0.0;
    for (int q = i; q < total && (ek[q] >> kSpPosBits) == row; ++q) sum += ev[ek[q] & ((1u << kSpPosBits) - 1)];
    adw[(size_t)row * w + g] = sum;
  }
}

int sparse_cs_smem() { return (2 * kBkSortCap + 1 + kSpCap) * 4 + 4 + kSpCap * 8; }

cudaError_t launch_sparse_countsketch(int dtype, const long long* cp, const int* ri, const void* val,
                                      long long n, const double* dvec, int is_d2, uint64_t seed, long long k,
                                      int retry, int s_blocks, int w, double* adw, int m, const CsWork& ws,
                                      int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(adw, 0, sizeof(double) * (size_t)m * w, st);
  if (e != cudaSuccess) return e;
  e = cs_lists(n, dvec, is_d2, seed, k, retry, s_blocks, w, ws, num_sms, st);
  if (e != cudaSuccess) return e;
  const int smem = sparse_cs_smem();
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (dtype == 0) {
    e = ensure_smem((const void*)k_sp_bucket<double>, smem);
    if (e != cudaSuccess) return e;
    k_sp_bucket<double><<<(unsigned)w, kSpThreads, smem, st>>>(cp, ri, static_cast<const double*>(val), w, ws.base,
                                                               ws.list, ws.sc64, adw);
  } else {
    e = ensure_smem((const void*)k_sp_bucket<float>, smem);
    if (e != cudaSuccess) return e;
    k_sp_bucket<float><<<(unsigned)w, kSpThreads, smem, st>>>(cp, ri, static_cast<const float*>(val), w, ws.base,
                                                              ws.list, ws.sc64, adw);
  }
  return cudaGetLastError();
}

cudaError_t launch_countsketch(int dtype, const void* A, int lda, int m, long long n,
                               const double* dvec, int is_d2, uint64_t seed, long long k,
                               int retry, int s_blocks, int w, double* adw, const CsWork& ws,
                               int* err, int num_sms, cudaStream_t st) {
  cudaError_t e = cs_lists(n, dvec, is_d2, seed, k, retry, s_blocks, w, ws, num_sms, st);
  if (e != cudaSuccess) return e;
  // the bucket kernel: whole columns through a ring of shared-memory stages
  const int esz = dtype == 0 ? 8 : (dtype == 1 ? 4 : 2);
  const int col_bytes = lda * esz;
  int rpt = 1;
  while (rpt * kBkRows < lda) rpt <<= 1;
  if (esz == 2) rpt = std::max(rpt, 2);
  const int stages = std::min(kBkMaxStages, kBkRingBytes / col_bytes) / 2 * 2;  // even: columns go in pairs
  // (columns of at most 512 rows go to the slab kernel, whose warps each take
  // whole columns: one element per thread and column would leave the bucket
  // kernel's consumers mostly waiting on the per-column handshake)
  if (lda > kBkRows && rpt <= 8 && stages >= 2) {
    const int bsmem = stages * col_bytes + kBkSortCap * (4 + 8) + 2 * stages * 8;
    auto go = [&](auto kern, const auto* a) -> cudaError_t {
      cudaError_t e2 = ensure_smem((const void*)kern, bsmem);
      if (e2 != cudaSuccess) return e2;
      g_launches.fetch_add(1, std::memory_order_relaxed);
      kern<<<(unsigned)w, kBkThreads, bsmem, st>>>(a, lda, m, w, stages, ws.base, ws.list, ws.sc64, ws.scdf,
                                                    adw, err);
      return cudaGetLastError();
    };
    if (dtype == 0) {
      const double* a = static_cast<const double*>(A);
      if (rpt == 1) return go(k_cs_bucket<double, 1>, a);
      if (rpt == 2) return go(k_cs_bucket<double, 2>, a);
      if (rpt == 4) return go(k_cs_bucket<double, 4>, a);
      return go(k_cs_bucket<double, 8>, a);
    }
    if (dtype == 1) {
      const float* a = static_cast<const float*>(A);
      if (rpt == 1) return go(k_cs_bucket<float, 1>, a);
      if (rpt == 2) return go(k_cs_bucket<float, 2>, a);
      if (rpt == 4) return go(k_cs_bucket<float, 4>, a);
      return go(k_cs_bucket<float, 8>, a);
    }
    const bf16raw* a = static_cast<const bf16raw*>(A);
    if (rpt == 2) return go(k_cs_bucket<bf16raw, 2>, a);
    if (rpt == 4) return go(k_cs_bucket<bf16raw, 4>, a);
    return go(k_cs_bucket<bf16raw, 8>, a);
  }
  // taller columns: one CTA per (bucket, 512-row slab), columns loaded by the warps
  // sorted keys + the warps' partial sums (FP64 or a double-float pair: 8 bytes)
  const int smem = kSortCap * (int)sizeof(int) + kAccWarps * kSlab * 8;
  dim3 grid((unsigned)w, (unsigned)((m + kSlab - 1) / kSlab));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (dtype == 0) {
    e = ensure_smem((const void*)k_cs_accum<double>, smem);
    if (e != cudaSuccess) return e;
    k_cs_accum<double><<<grid, kAccThreads, smem, st>>>(static_cast<const double*>(A), lda, m, w, ws.base,
                                                         ws.list, ws.sc64, ws.scdf, adw);
  } else if (dtype == 1) {
    e = ensure_smem((const void*)k_cs_accum<float>, smem);
    if (e != cudaSuccess) return e;
    k_cs_accum<float><<<grid, kAccThreads, smem, st>>>(static_cast<const float*>(A), lda, m, w, ws.base,
                                                        ws.list, ws.sc64, ws.scdf, adw);
  } else {
    e = ensure_smem((const void*)k_cs_accum<bf16raw>, smem);
    if (e != cudaSuccess) return e;
    k_cs_accum<bf16raw><<<grid, kAccThreads, smem, st>>>(static_cast<const bf16raw*>(A), lda, m, w, ws.base,
                                                          ws.list, ws.sc64, ws.scdf, adw);
  }
  return cudaGetLastError();
}

cudaError_t launch_v_gather(long long n, const double* x, const double* s, const double* u,
                            uint64_t seed, long long k, int retry, int s_blocks, int w, double scale,
                            double* v, int num_sms, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_v_gather<<<grid, 256, 0, st>>>(n, x, s, u, seed, k, retry, s_blocks, w / s_blocks, scale, v);
  return cudaGetLastError();
}

}  // namespace lpk
