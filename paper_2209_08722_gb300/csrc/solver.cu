// Host driver of the GB300 sketched inexact IPM: the C ABI of lp_sketch_ipm.h.
//
// Outer iteration (Algorithm 3 step numbers; Algorithm 2 is the same with
// r_d = 0 and p from eq. pdef):
//   step 3   one FP64 A-pass: r_p = A x - b, r_d = A^T y + s - c, p, d^2
//   step 2   CountSketch A D W (sketch.cu)
//   Alg. 1   QR of (ADW)^T (cuSOLVER geqrf) and R^{-1} (cuSOLVER trtri):
//            Q = A D W W^T D A^T = R^T R, Q^{-1} = R^{-1} R^{-T}
//   step 4   PCG on eq. (precond) with preconditioner Q^{-1}: FP32 products
//            (k_adat_fused), FP64 true-residual refresh every `refine_every`
//            steps, stop at ||f|| = sqrt(r^T Q^{-1} r) <= tol (Lemma 4.4)
//   step 5   v of eq. (compv) = (XS)^{1/2} W (ADW)^T Q^{-1} (M dy - p)
//            (using (ADW)^+ = (ADW)^T Q^{-1} for full row rank), the
//            directions (one FP64 A^T-pass), then the step lengths (steps 6-7)
//            and the update (step 8).
// The host synchronises a few times per outer iteration (stopping test, rank
// check, inner-solve chunks); everything else is stream-ordered.
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <system_error>
#include <string>
#include <vector>

#include "../../include/lp_sketch_ipm.h"
#include "host_math.h"
#include "internal.h"

#include <atomic>
#include <map>
#include <mutex>
#include <thread>

using namespace lpk;

namespace {
// per host thread, so that threads creating handles at once do not race on it
thread_local std::string g_create_error;

long long round_up_ll(long long x, long long a) { return (x + a - 1) / a * a; }

struct EvPair {
  cudaEvent_t a, b;
};

// A matrix given by rows (CSR) in the column form the sparse kernels stream
// (CSC), built on the host by a counting sort on the column index: one pass
// counts each column's entries, a prefix sum gives the column pointers, and a
// second pass over the rows in order places every entry, so each column's
// entries come out in increasing row order (a stable sort: the result depends
// only on the matrix).  Returns an empty string, or the structural error found
// in the CSR arrays (row pointers not starting at 0, decreasing, or not ending
// at nnz; a column index outside [0, n)).
//
// Large matrices are sorted in parts: the rows are split into contiguous
// ranges of about equal entry counts, each part counts its own entries per
// column, and within a column the parts take their slots in row order, so the
// result is the serial sort's, bit for bit, whatever the number of parts.
struct CscCopy {
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
  std::vector<char> val;
};

// f(t) for t in [0, parts): parts 1.. on worker threads, part 0 (and any part
// whose thread cannot be started) on the calling thread.  f must not throw.
template <typename F>
void run_parts(int parts, const F& f) {
  std::vector<std::thread> workers;
  workers.reserve((size_t)parts);
  std::vector<int> here;
  here.reserve((size_t)parts);
  for (int t = 1; t < parts; ++t) {
    try {
      workers.emplace_back(f, t);
    } catch (...) {
      here.push_back(t);
    }
  }
  f(0);
  for (int t : here) f(t);
  for (auto& w : workers) w.join();
}

// V: an unsigned integer of the element's size (values are moved bit for bit)
template <typename V>
void csr_to_csc_fill(int m, long long n, long long nnz, const int64_t* rp, const int32_t* ci, const V* v,
                     CscCopy* out) {
  // parts: at most 8 and the host's threads, none for small matrices, and at
  // most 256 MB of per-part column slots
  int parts = (int)std::min<unsigned>(8u, std::max(1u, std::thread::hardware_concurrency()));
  if (nnz < (1LL << 20) || m < 2 * parts) parts = 1;
  while (parts > 1 && (double)parts * (double)n * sizeof(int64_t) > 256e6) --parts;
  std::vector<int> rb((size_t)parts + 1);
  rb[0] = 0;
  rb[parts] = m;
  for (int t = 1; t < parts; ++t) {
    const long long target = nnz / parts * t;
    rb[t] = std::max(rb[t - 1], (int)(std::lower_bound(rp, rp + m + 1, (int64_t)target) - rp));
    rb[t] = std::min(rb[t], m);
  }
  // slot[t][j]: part t's count in column j, then its next free slot there
  std::vector<int64_t> slot((size_t)parts * n, 0);
  run_parts(parts, [&](int t) {
    int64_t* c = slot.data() + (size_t)t * n;
    for (long long q = rp[rb[t]]; q < rp[rb[t + 1]]; ++q) ++c[ci[q]];
  });
  out->ptr.assign((size_t)n + 1, 0);
  int64_t run = 0;
  for (long long j = 0; j < n; ++j) {
    out->ptr[j] = run;
    for (int t = 0; t < parts; ++t) {
      int64_t& c = slot[(size_t)t * n + j];
      const int64_t k = c;
      c = run;
      run += k;
    }
  }
  out->ptr[n] = run;
  out->idx.resize((size_t)std::max<long long>(nnz, 1));
  out->val.resize((size_t)std::max<long long>(nnz, 1) * sizeof(V));
  int32_t* idx = out->idx.data();
  V* val = reinterpret_cast<V*>(out->val.data());
  run_parts(parts, [&](int t) {
    int64_t* c = slot.data() + (size_t)t * n;
    for (int i = rb[t]; i < rb[t + 1]; ++i)
      for (long long q = rp[i]; q < rp[i + 1]; ++q) {
        const int64_t dst = c[ci[q]]++;
        idx[dst] = i;
        val[dst] = v[q];
      }
  });
}

std::string csr_to_csc(int m, long long n, long long nnz, const int64_t* rp, const int32_t* ci,
                       const void* val, int esz, CscCopy* out) {
  if (rp[0] != 0 || rp[m] != nnz) return "CSR ptr[0] != 0 or ptr[m] != nnz";
  for (int i = 0; i < m; ++i)
    if (rp[i + 1] < rp[i]) return "CSR row pointers not monotone";
  for (long long q = 0; q < nnz; ++q)
    if (ci[q] < 0 || ci[q] >= n) return "CSR column index out of range";
  if (esz == 8) csr_to_csc_fill(m, n, nnz, rp, ci, static_cast<const uint64_t*>(val), out);
  else if (esz == 4) csr_to_csc_fill(m, n, nnz, rp, ci, static_cast<const uint32_t*>(val), out);
  else csr_to_csc_fill(m, n, nnz, rp, ci, static_cast<const uint16_t*>(val), out);
  return std::string();
}
}  // namespace

// Device blocks freed by destroyed handles are kept for the next handles
// (keyed by device and size), up to kPoolCap bytes: a handle of a shape
// solved before is then created without cudaMalloc and destroyed without
// cudaFree, which for large A is most of its creation and destruction time.
// A failed cudaMalloc empties the cache and retries; lp_release_cached_memory
// returns the cache to the driver.
namespace {
constexpr size_t kPoolCap = size_t(16) << 30;
std::mutex g_pool_mu;
std::multimap<std::pair<int, size_t>, void*> g_pool;
size_t g_pool_bytes = 0;

void* pool_take(int dev, size_t bytes) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  auto it = g_pool.find({dev, bytes});
  if (it == g_pool.end()) return nullptr;
  void* p = it->second;
  g_pool.erase(it);
  g_pool_bytes -= bytes;
  return p;
}

void pool_give(int dev, size_t bytes, void* p) {
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool_bytes + bytes <= kPoolCap) {
      g_pool.insert({{dev, bytes}, p});
      g_pool_bytes += bytes;
      return;
    }
  }
  cudaFree(p);
}

void pool_release() {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (auto& kv : g_pool) cudaFree(kv.second);
  g_pool.clear();
  g_pool_bytes = 0;
}
}  // namespace

struct lp_handle {
  int dev = 0, num_sms = 1;
  int m = 0;
  long long n = 0, npad = 0;
  int lda = 0, dtype = 0, esz = 0, fmt = 0;
  void* A = nullptr;
  lp_options opt{};
  int w = 0, s_blocks = 2;
  double bnorm = 0.0, cnorm = 0.0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  // second stream and events for the factor's overlapped pivot kernels (sweep.cu)
  cudaStream_t st_aux = nullptr;
  cudaEvent_t ev_x = nullptr, ev_p = nullptr;
  // phase timing without host synchronisation: the correction and step phases
  // of an outer iteration are bracketed by these, read after the next
  // synchronisation
  cudaEvent_t ev_cor = nullptr, ev_step = nullptr, ev_end = nullptr, ev_res = nullptr, ev_res_end = nullptr;
  cusolverDnHandle_t sol = nullptr;
  cublasHandle_t blas = nullptr;
  int lwork_potrf = 0;
  long long qr_fallbacks = 0;
  long long cheb_fallbacks = 0;
  bool use_df = false;   // double-float kernel for the FP64-accurate products
  bool use_df_resid = false, use_df_dir = false;  // ... and for the residual / direction passes
  float2* dfin[4] = {nullptr, nullptr, nullptr, nullptr};  // packed per-column inputs
  float2* dfout[2] = {nullptr, nullptr};                   // per-column outputs as pairs
  float2* d2df = nullptr;  // d2 as pairs for the double-float refresh
  float2* cdf = nullptr;   // c as pairs (constant)
  bool d2df_valid = false;
  bool sparse = false;   // CSC storage
  const double* sk_dvec = nullptr;  // D (or D^2) used by the current sketch
  int sk_is_d2 = 0;
  long long* colptr = nullptr;
  int* rowidx = nullptr;
  void* spval = nullptr;
  long long nnz = 0;
  int sp_grid = 0;
  // the same sparse A by rows, in row segments, for the two-pass kernels
  long long* rowptr = nullptr;
  int* colidx = nullptr;
  void* rval = nullptr;
  long long* seg = nullptr;
  int* seg_row = nullptr;
  int* row_seg = nullptr;
  int nseg = 0;
  double* tcol = nullptr;
  double* segsum = nullptr;
  bool qinv_ok = false;  // explicit Q^{-1} formed for the current factor
  double* qinv = nullptr;
  bool qinv_df_ok = false;  // ... and as FP32 pairs (the sweep's output), for the double-float GEMV
  float2* qinv_df = nullptr;
  CsWork cs;             // CountSketch bucket lists and scales (dense, and sparse where they fit)
  float* gram_scratch = nullptr;  // double-float Gram: split ADW + split-K partials
  float* sweep_scratch = nullptr; // double-float sweep: two m x m iterates + pivots
  long long sweep_fallbacks = 0;
  long long breakdown_recoveries = 0;  // inner solves that switched product after a CG breakdown
  long long qr_refactors = 0;          // inner solves rerun after refactoring by QR
  long long poor_redraws = 0;          // draws of W replaced after failing the Ritz check
  long long indefinite_refactors = 0;  // FP64 refactors after r^T Q^{-1} r <= 0
  int factor_kind = 0;  // factor in use: 0 double-float sweep, 1 FP64 Cholesky, 2 FP64 QR
  double ratio_ref = 0.0;  // largest accepted max/min |R_ii| of this solve (0: none yet)
  long long jump_redraws = 0;  // draws of W replaced after a jump of max/min |R_ii|
  double *dy_aff = nullptr, *dy_c = nullptr, *p_aff = nullptr, *p_c = nullptr;  // two-RHS variant (m)
  double *v_aff = nullptr, *v_c = nullptr;                                        // ... (n)
  // learned / previous-direction warm start of the inner solve
  int ws_mode = 0;
  lp_mlp* ws_model = nullptr;
  float *ws_rec_X = nullptr, *ws_rec_T = nullptr;
  long long ws_cap = 0, ws_count = 0, ws_props = 0, ws_acc = 0;
  bool ws_have_prev = false;
  double *dy_prev = nullptr, *ws_u = nullptr;
  double *ws_v = nullptr, *ws_w = nullptr, *ws_dots = nullptr;  // proposal, M v_i (2 m), dots
  bool warm_r_ready = false;  // h->r already holds p - M dy^0 for the warm start
  float *ws_X = nullptr, *ws_Y = nullptr;
  float* ws_hid = nullptr;  // the model's activations and GEMV partials (per handle)
  long long ws_hid_cap = 0;
  // n-vectors (padded)
  double *c = nullptr, *x = nullptr, *y = nullptr, *s = nullptr, *rd = nullptr, *d2d = nullptr,
         *dx = nullptr, *ds = nullptr, *v = nullptr, *nb0 = nullptr, *nb1 = nullptr, *nb2 = nullptr;
  float* d2f = nullptr;
  // m-vectors
  double *b = nullptr, *rp = nullptr, *p = nullptr, *dy = nullptr, *r = nullptr, *z = nullptr,
         *pdir = nullptr, *q = nullptr, *wv = nullptr, *mb0 = nullptr, *mb1 = nullptr;
  double* coef = nullptr;  // CG coefficients for the Lanczos interval
  // sketch and factor
  double *adw = nullptr, *qr = nullptr, *tau = nullptr, *rinv_cm = nullptr, *rinv_rm = nullptr,
         *uw = nullptr, *adwt_part = nullptr;
  int adwt_parts = 64;
  void* dwork = nullptr;
  size_t dwork_bytes = 0;
  void* hwork = nullptr;
  size_t hwork_bytes = 0;
  int lwork_geqrf = 0;
  int* dinfo = nullptr;
  // scratch
  void* partials = nullptr;
  double* gpart = nullptr;
  unsigned* gtickets = nullptr;
  double* red_partials = nullptr;
  unsigned* tickets = nullptr;
  double* vpart = nullptr;
  DevScalars* sc = nullptr;
  DevScalars* hsc = nullptr;  // pinned host copy
  int* hinfo = nullptr;       // pinned
  double* hval = nullptr;     // pinned staging for scalars
  StreamPlan plan;
  // CUDA graphs of one block of inner steps (refine_every products and
  // preconditioner GEMVs, then the true-residual refresh), captured once per
  // handle and variant (inner method, form of the stored preconditioner) and
  // replayed with one launch per block
  struct BlockGraph {
    cudaGraphExec_t exec = nullptr;
    int key = -1;
    long long kernels = 0;
  };
  BlockGraph blk_graph[2];
  bool graphs_failed = false;
  long long graph_replays = 0;
  StreamPlan fplan;        // tile plan of the warp-per-column FP32 product (opt.autotune may change it)
  bool prod_rows = false;  // the FP32 product uses the row-split kernel
  int alloc_grid = 0;      // CTAs the per-CTA partial buffers were sized for
  RowsPlan rplan;          // row-split kernels for tall columns (stream_rows.cu): FP32 product
  RowsPlan rplan_df;       // ... and the double-float passes
  bool use_rows = false;   // the FP32 product and the double-float passes use them
  std::string err;
  // profiling of the hot product kernel
  std::vector<EvPair> ev_pool;
  size_t ev_used = 0;
  long long k1_launches = 0;
  double k1_ms = 0.0;
  unsigned long long k1_sample = 0;  // product launches seen by the profiling sampler
  long long launch_base = 0;
  std::vector<lp_iter_record> history;
  std::vector<std::pair<void*, size_t>> allocs;  // device blocks and their sizes
  // checkpoint / resume: the state of the last solve (valid while x, y, s
  // still hold its iterate) and a state loaded for the next solve
  bool state_valid = false;
  lp_state last_state{};
  bool resume_pending = false;
  lp_state resume{};

  int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  // opt.guard: guard regions of kGuard bytes of kGuardByte on both sides of
  // every buffer (the user part stays 256-byte aligned)
  static constexpr size_t kGuard = 256;
  static constexpr unsigned char kGuardByte = 0xA5;
  struct GuardedBuf {
    char* base;
    size_t bytes;
  };
  std::vector<GuardedBuf> guarded_bufs;
  template <typename T>
  int alloc(T** ptr, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    const size_t pad = opt.guard ? kGuard : 0;
    const size_t total = bytes + 2 * pad;
    void* p = pool_take(dev, total);
    if (!p && cudaMalloc(&p, total) != cudaSuccess) {
      cudaGetLastError();
      pool_release();  // the cached blocks may be what the device is short of
      if (cudaMalloc(&p, total) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(LP_ERR_OOM, "cudaMalloc of %zu bytes failed", total);
      }
    }
    allocs.push_back({p, total});
    char* user = static_cast<char*>(p) + pad;
    if (pad) {
      guarded_bufs.push_back({static_cast<char*>(p), bytes});
      cudaMemsetAsync(p, kGuardByte, pad, st);
      cudaMemsetAsync(user + bytes, kGuardByte, pad, st);
    }
    cudaMemsetAsync(user, 0, bytes, st);
    *ptr = reinterpret_cast<T*>(user);
    return LP_OK;
  }
  cudaStream_t stream() const { return st; }
};

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) return h->fail(LP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
  } while (0)
#define CS(call)                                                                       \
  do {                                                                                 \
    cusolverStatus_t _s = (call);                                                      \
    if (_s != CUSOLVER_STATUS_SUCCESS) return h->fail(LP_ERR_CUDA, "%s: status %d", #call, (int)_s); \
  } while (0)
#define RET(call)              \
  do {                         \
    int _r = (call);           \
    if (_r < 0) return _r;     \
  } while (0)

namespace {

// the device status word of the last copy of the scalars, as an error code
int check_read(lp_handle* h) {
  if (h->hsc->err == ERR_TIMEOUT) return h->fail(LP_ERR_DEVICE_TIMEOUT, "device wait timed out");
  if (h->hsc->err == ERR_NUMERICAL) return h->fail(LP_ERR_NUMERICAL, "non-finite value in a reduction");
  return LP_OK;
}

int sync_read(lp_handle* h) {
  CK(cudaMemcpyAsync(h->hsc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return check_read(h);
}

// A call starts from a clear device status word, so that an error reported by
// an earlier call (a wait that gave up, a non-finite reduction) does not stick
// to the handle.
int clear_status(lp_handle* h) {
  CK(cudaMemsetAsync(&h->sc->err, 0, sizeof(int), h->st));
  return LP_OK;
}

int set_scalar(lp_handle* h, double* dev_field, double value) {
  CK(cudaStreamSynchronize(h->st));
  *h->hval = value;
  CK(cudaMemcpyAsync(dev_field, h->hval, sizeof(double), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return LP_OK;
}

StreamArgs base_args(lp_handle* h) {
  StreamArgs a;
  std::memset(&a, 0, sizeof a);
  a.A = h->A;
  a.lda = h->lda;
  a.m = h->m;
  a.n = h->n;
  a.nb = h->plan.nb;
  a.ntiles = h->plan.ntiles;
  a.stages = h->plan.stages;
  a.sigma = h->opt.sigma;
  a.partials = h->partials;
  a.gpart = h->gpart;
  a.gtickets = h->gtickets;
  a.colptr = h->colptr;
  a.rowidx = h->rowidx;
  a.spval = h->spval;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.rval = h->rval;
  a.seg = h->seg;
  a.seg_row = h->seg_row;
  a.row_seg = h->row_seg;
  a.nseg = h->nseg;
  a.tcol = h->tcol;
  a.segsum = h->segsum;
  a.ticket = h->tickets + 0;
  a.sc = h->sc;
  a.err = &h->sc->err;
  return a;
}

// ---- profiling of the hot product (opt.profile) ----
EvPair* ev_next(lp_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    EvPair e;
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return &h->ev_pool[h->ev_used++];
}

void ev_flush(lp_handle* h) {
  for (size_t i = 0; i < h->ev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[i].a, h->ev_pool[i].b) == cudaSuccess) {
      h->k1_ms += ms;
      h->k1_launches += 1;
    }
  }
  h->ev_used = 0;
}

// u = A diag(d2) A^T v with FP32 products (the hot kernel) or FP64
int launch_adat(lp_handle* h, const double* vin, int epilogue, bool fp64, int skip_level,
                double* out_m0) {
  StreamArgs a = base_args(h);
  const bool use64 = fp64 || h->dtype == LP_F64;
  const bool dfk = use64 && !h->sparse && h->use_df;
  if (dfk && !h->d2df_valid) {
    DfPackArgs pk{{h->d2d}, {h->d2df}, 1, h->n};
    CK(launch_df_pack(pk, h->num_sms, h->st));
    h->d2df_valid = true;
  }
  a.cv[0] = dfk ? (const void*)h->d2df : (use64 ? (const void*)h->d2d : (const void*)h->d2f);
  a.cv_esz[0] = use64 ? 8 : 4;
  a.ncv = 1;
  a.vin = vin;
  a.epilogue = epilogue;
  a.skip_level = skip_level;
  a.out_m0 = out_m0;
  a.pcg_p = h->pdir;
  a.pcg_r = h->r;
  a.pcg_dy = h->dy;
  a.bvec = h->p;
  a.coef = h->coef;
  // Inner-loop products (skip_level 1) and their GEMVs use programmatic
  // dependent launch, which hides most of the launch latency between the two.
  // With opt.profile, one run of 8 FP32 products in 8 (a whole block of CG
  // steps) is launched plainly, and so are its GEMVs (events between the
  // kernels would stop the overlap, and a single plain launch among
  // overlapped ones would be timed with its dispatch); its products after the
  // first (which follows a host synchronisation) are timed between CUDA
  // events. The other blocks keep the overlap.
  EvPair* ev = nullptr;
  bool pdl = skip_level == 1 && !use64;
  if (h->opt.profile && !use64) {
    const unsigned long long k = h->k1_sample++;
    if (((k >> 3) & 7) == 0) {
      pdl = false;
      if ((k & 7) != 0) {
        ev = ev_next(h);
        if (ev) cudaEventRecord(ev->a, h->st);
      }
    }
  }
  cudaError_t e;
  if (h->sparse) e = launch_sparse2(h->dtype, use64, M_ADAT, a, h->num_sms, h->st);
  else if (!use64 && h->prod_rows) e = launch_rows(h->dtype, false, M_ADAT, a, h->rplan, h->st, pdl);
  else if (!use64) {
    a.nb = h->fplan.nb;
    a.ntiles = h->fplan.ntiles;
    a.stages = h->fplan.stages;
    e = launch_adat_fused(h->dtype, a, h->fplan, h->st, pdl);
  }
  else if (h->use_rows) {
    // the refresh inside the inner loop follows a GEMV closely
    e = launch_rows(h->dtype, true, M_ADAT, a, h->rplan_df, h->st, skip_level >= 1);
  } else if (h->use_df) {
    a.pdl = skip_level >= 1 ? 1 : 0;  // the refresh inside the inner loop follows a GEMV closely
    e = launch_stream_df(h->dtype, M_ADAT, a, h->plan, h->st);
  }
  else e = launch_stream(h->dtype, true, M_ADAT, a, h->plan, h->st);
  if (ev) cudaEventRecord(ev->b, h->st);
  if (e != cudaSuccess) return h->fail(LP_ERR_CUDA, "adat launch: %s", cudaGetErrorString(e));
  return LP_OK;
}

int precond_gemvs(lp_handle* h, const double* r, double* z, int epi, int skip_level) {
  // inner-loop GEMVs follow their product closely (see launch_adat); those of
  // a block sampled by opt.profile are launched plainly, like its products
  const bool pdl = skip_level >= 1 && !(h->opt.profile && (((h->k1_sample - 1) >> 3) & 7) == 0);
  if (!h->opt.precondition) {  // Q = I: z = r, then the same CG / Chebyshev epilogue
    cudaError_t e = launch_gemv_tri(nullptr, h->m, 2, r, z, epi, skip_level, h->r, h->pdir, h->dy, h->sc,
                                    h->tickets + 2, &h->sc->err, h->opt.t_max, h->coef, h->num_sms, h->st,
                                    nullptr, nullptr, pdl);
    if (e != cudaSuccess) return h->fail(LP_ERR_CUDA, "gemv: %s", cudaGetErrorString(e));
    return LP_OK;
  }
  if (h->qinv_ok) {  // one full GEMV with the explicit Q^{-1} (as pairs when the sweep formed it)
    cudaError_t e = launch_gemv_tri(h->qinv, h->m, 2, r, z, epi, skip_level, h->r, h->pdir, h->dy,
                                    h->sc, h->tickets + 2, &h->sc->err, h->opt.t_max, h->coef,
                                    h->num_sms, h->st, nullptr, h->qinv_df_ok ? h->qinv_df : nullptr, pdl);
    if (e != cudaSuccess) return h->fail(LP_ERR_CUDA, "gemv: %s", cudaGetErrorString(e));
    return LP_OK;
  }
  cudaError_t e = launch_gemv_tri(h->rinv_cm, h->m, 1, r, h->wv, GH_NONE, skip_level, nullptr,
                                  nullptr, nullptr, h->sc, h->tickets + 1, &h->sc->err, 0, nullptr,
                                  h->num_sms, h->st, nullptr, nullptr, pdl);
  if (e != cudaSuccess) return h->fail(LP_ERR_CUDA, "gemv: %s", cudaGetErrorString(e));
  e = launch_gemv_tri(h->rinv_rm, h->m, 0, h->wv, z, epi, skip_level, h->r, h->pdir, h->dy, h->sc,
                      h->tickets + 2, &h->sc->err, h->opt.t_max, h->coef, h->num_sms, h->st, nullptr,
                      nullptr, pdl);
  if (e != cudaSuccess) return h->fail(LP_ERR_CUDA, "gemv: %s", cudaGetErrorString(e));
  return LP_OK;
}

// Q^{-1} = R^{-1} R^{-T} (cuBLAS DSYRK on the explicit R^{-1}, then mirrored),
// so each CG step applies the preconditioner with one GEMV.
int form_qinv(lp_handle* h) {
  h->qinv_ok = false;
  if (!h->blas) return LP_OK;
  const int m = h->m;
  const double one = 1.0, zero = 0.0;
  if (cublasDsyrk(h->blas, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, m, m, &one, h->rinv_cm, m, &zero,
                  h->qinv, m) != CUBLAS_STATUS_SUCCESS)
    return LP_OK;  // keep the two triangular GEMVs
  CK(launch_factor_utils(3, h->qinv, m, m, h->qinv, h->sc, 0.0, h->num_sms, h->st));
  h->qinv_ok = true;
  return LP_OK;
}

// QR of (ADW)^T and R^{-1}; LP_ERR_SKETCH_RANK on a rank failure.
int factor_qr(lp_handle* h);

// Cholesky of the Gram left in rinv_cm (upper triangle) by cuSOLVER potrf,
// R^{-1} by trtri and Q^{-1} = R^{-1} R^{-T}; the fallback of the sweep.
int factor_chol(lp_handle* h) {
  const int m = h->m, w = h->w;
  CS(cusolverDnDpotrf(h->sol, CUBLAS_FILL_MODE_UPPER, m, h->rinv_cm, m,
                      static_cast<double*>(h->dwork), h->lwork_potrf, h->dinfo));
  CK(launch_factor_utils(0, h->rinv_cm, m, m, h->rinv_cm, h->sc, 0.0, h->num_sms, h->st));
  CK(launch_factor_utils(1, h->rinv_cm, m, m, nullptr, h->sc, 1e-13, h->num_sms, h->st));
  CK(cudaMemcpyAsync(h->hinfo, h->dinfo, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  RET(sync_read(h));
  if (h->hinfo[0] == 0 && !h->hsc->rank_bad) {
    CS(cusolverDnXtrtri(h->sol, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, m, CUDA_R_64F,
                        h->rinv_cm, m, h->dwork, h->dwork_bytes, h->hwork, h->hwork_bytes,
                        h->dinfo + 1));
    CK(launch_factor_utils(2, h->rinv_cm, w, m, h->rinv_rm, h->sc, 0.0, h->num_sms, h->st));
    CK(cudaMemcpyAsync(h->hinfo + 1, h->dinfo + 1, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    RET(sync_read(h));
    if (h->hinfo[1] == 0) {
      h->factor_kind = 1;
      return form_qinv(h);
    }
  }
  h->qr_fallbacks += 1;
  return factor_qr(h);
}

// Q = (ADW)(ADW)^T by a Gram in double-float arithmetic (FP64-class accuracy
// on the FP32 pipe, gram.cu) and Q^{-1} directly by the blocked symmetric
// sweep (sweep.cu), whose pivots give the rank check.  The Gram squares
// kappa(ADW), which stays far below the inverse unit roundoff on the IPM path;
// if a pivot is not safely positive, the FP64 Cholesky of the same Gram and
// then the QR of (ADW)^T are tried.
int factor(lp_handle* h) {
  const int m = h->m, w = h->w;
  h->qinv_ok = false;
  CK(launch_gram_df(h->adw, m, w, h->gram_scratch, h->rinv_cm, h->num_sms, h->st));
  h->qinv_df_ok = false;
  // Q^{-1} is kept as pairs only: the double-float GEMV applies it
  CK(launch_sweep_inverse(h->rinv_cm, m, h->sweep_scratch, nullptr, h->qinv_df, h->sc, 1e-13, h->num_sms,
                          h->st, h->st_aux, h->ev_x, h->ev_p));
  RET(sync_read(h));
  if (!h->hsc->rank_bad) {
    h->qinv_ok = true;
    h->qinv_df_ok = true;
    h->factor_kind = 0;
    return LP_OK;
  }
  h->sweep_fallbacks += 1;
  if (h->blas) return factor_chol(h);
  return factor_qr(h);
}

// Q = R^T R from the QR of (ADW)^T (cuSOLVER geqrf), R^{-1} by trtri.
int factor_qr(lp_handle* h) {
  const int m = h->m, w = h->w;
  h->qinv_ok = false;
  h->qinv_df_ok = false;
  CK(cudaMemcpyAsync(h->qr, h->adw, sizeof(double) * (size_t)m * w, cudaMemcpyDeviceToDevice, h->st));
  CS(cusolverDnDgeqrf(h->sol, w, m, h->qr, w, h->tau, static_cast<double*>(h->dwork),
                      h->lwork_geqrf, h->dinfo));
  CK(launch_factor_utils(0, h->qr, w, m, h->rinv_cm, h->sc, 0.0, h->num_sms, h->st));
  CK(launch_factor_utils(1, h->rinv_cm, w, m, nullptr, h->sc, 1e-13, h->num_sms, h->st));
  CS(cusolverDnXtrtri(h->sol, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, m, CUDA_R_64F,
                      h->rinv_cm, m, h->dwork, h->dwork_bytes, h->hwork, h->hwork_bytes,
                      h->dinfo + 1));
  CK(launch_factor_utils(2, h->rinv_cm, w, m, h->rinv_rm, h->sc, 0.0, h->num_sms, h->st));
  CK(cudaMemcpyAsync(h->hinfo, h->dinfo, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  RET(sync_read(h));
  if (h->hsc->rank_bad || h->hinfo[0] != 0 || h->hinfo[1] != 0)
    return h->fail(LP_ERR_SKETCH_RANK, "A D W is numerically rank deficient (|R_ii| range %.3e..%.3e)",
                   h->hsc->diag_min, h->hsc->diag_max);
  h->factor_kind = 2;
  return form_qinv(h);
}

// A D W for the sketch of (seed, k, retry): Gaussian (dense A) or CountSketch
// (dense or CSC).  Remembers which D it used, for the correction vector.
cudaError_t launch_sketch(lp_handle* h, const double* dvec, int is_d2, uint64_t seed, long long k,
                          int retry) {
  h->sk_dvec = dvec;
  h->sk_is_d2 = is_d2;
  if (h->opt.sketch == LP_SKETCH_GAUSS)
    return launch_gauss_sketch(h->dtype, h->A, h->lda, h->m, h->n, dvec, is_d2, seed, k, retry, h->w,
                               h->adw, h->opt.tensor_sketch, &h->sc->err, h->num_sms, h->st);
  if (h->sparse && h->cs.list)
    return launch_sparse_countsketch(h->dtype, h->colptr, h->rowidx, h->spval, h->n, dvec, is_d2, seed, k,
                                     retry, h->s_blocks, h->w, h->adw, h->m, h->cs, h->num_sms, h->st);
  if (h->sparse)
    return launch_sparse_sketch(h->dtype, h->colptr, h->rowidx, h->spval, h->n, dvec, is_d2, seed, k,
                                retry, h->s_blocks, h->w, h->adw, h->m, h->num_sms, h->st);
  return launch_countsketch(h->dtype, h->A, h->lda, h->m, h->n, dvec, is_d2, seed, k, retry,
                            h->s_blocks, h->w, h->adw, h->cs, &h->sc->err, h->num_sms, h->st);
}

// Largest jump of max/min |R_ii| (a lower bound on kappa(A D W)) over the
// largest accepted value of the solve that a draw may show.  On the central path
// kappa(A D) grows smoothly (about 2.5x per outer iteration at most on the
// planted families); near the optimum range((AD)^T) is close to the span of the
// m basic coordinates, and a draw whose rows for those columns are linearly
// dependent (with s = 2: two columns sharing both buckets, or a cycle of
// shared buckets with the wrong sign parity) leaves only the nonbasic columns,
// about (mu / x_B)^{1/2} times smaller, to fill the lost direction: the ratio
// jumps by 1e4 or more in one iteration (the double-float Gram's rounding
// floor can hide part of the jump from the sweep's pivots).
constexpr double kRatioJump = 1e2;
constexpr int kJumpRedraws = 6;

// sketch for (k, retry) + factor, redrawing (retry + 1) on a rank failure
// (Lemma 4.1) and, within a solve, on a jump of max/min |R_ii| (above).
// *retries holds the first retry index to try and receives the one in use.
int sketch_and_factor(lp_handle* h, const double* dvec, int is_d2, long long k, int* retries) {
  if (!h->opt.precondition) {  // the unpreconditioned comparison: no sketch, no factor
    *retries = 0;
    return LP_OK;
  }
  int rc = LP_ERR_SKETCH_RANK;
  int jumps = 0;
  for (int retry = *retries; retry < kMaxRetry; ++retry) {
    CK(launch_sketch(h, dvec, is_d2, h->opt.seed, k, retry));
    rc = factor(h);
    *retries = retry;
    if (rc == LP_ERR_SKETCH_RANK) continue;
    if (rc != LP_OK) return rc;
    const double ratio = h->hsc->diag_min > 0 ? h->hsc->diag_max / h->hsc->diag_min : INFINITY;
    if (h->ratio_ref > 0.0 && ratio > kRatioJump * h->ratio_ref && jumps < kJumpRedraws &&
        retry + 1 < kMaxRetry) {
      jumps += 1;
      h->jump_redraws += 1;
      continue;
    }
    if (ratio <= kRatioJump * h->ratio_ref || h->ratio_ref == 0.0)
      h->ratio_ref = std::max(h->ratio_ref, ratio);
    return LP_OK;
  }
  return rc;
}

// Extreme Ritz values of Q^{-1} M from the first kk CG steps: the Lanczos
// tridiagonal has diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal
// sqrt(beta_j)/alpha_j (alpha_j at coef[2j], beta_j at coef[2j+1]).
// (lanczos_extremes in host_math.h; a broken recurrence keeps the defaults)
int ritz_extremes(lp_handle* h, int kk, double* lo, double* hi) {
  *lo = 0.5;
  *hi = 2.0;
  if (kk <= 0) return LP_OK;
  std::vector<double> coef(2 * (size_t)kk);
  CK(cudaMemcpyAsync(coef.data(), h->coef, sizeof(double) * 2 * kk, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  lanczos_extremes(coef.data(), kk, lo, hi);
  return LP_OK;
}

// Inner-solve status (never returned to the caller of the library): the first
// CG steps show Q^{-1} M with a spread far beyond what an embedding of eq.
// pdprec allows, i.e. this draw of W is one of the probability-delta failures
// of Lemma 4.1, and the solve has not converged.
constexpr int kInnerSketchPoor = 100;
// Inner-solve status: r^T Q^{-1} r <= 0 for r != 0 (inner_done = 3), i.e. the
// stored Q^{-1} is not positive definite at this residual.  The double-float
// sweep inverts the Gram by Gauss-Jordan, whose error relative to ||Q^{-1}|| is
// about kappa(Q) u; once that exceeds 1 / kappa(Q) the stored inverse can be
// indefinite.  Q^{-1} = R^{-1} R^{-T} from an FP64 Cholesky or QR is the Gram
// of R^{-1} and keeps its definiteness up to kappa(Q) ~ 1 / u_64.
constexpr int kInnerIndefinite = 101;
constexpr double kRitzSpread = 1e3;  // ((1 + e)/(1 - e))^2 = 1e3 at e ~ 0.94
constexpr int kPoorCheckIters = 32;  // act only on solves still running here ...
constexpr double kRitzSevere = 1e6;  // ... or at once beyond this spread

// One block of inner steps on the stream: `refine` steps of CG (or
// Chebyshev), each a product and the preconditioner GEMV with the method's
// epilogue, then the FP64-class true residual r = p - M dy and its GEMV.
// Every kernel skips its work on the device once the solve has converged
// (skip levels 1 and 2), so the block's launches do not depend on the state.
int enqueue_cg_block(lp_handle* h, int inner, bool use64, int refine) {
  const int m = h->m;
  for (int j = 0; j < refine; ++j) {
    if (inner == LP_INNER_CHEBYSHEV) {
      CK(launch_cheb_pre(m, h->dy, h->pdir, h->sc, h->st));
      RET(launch_adat(h, h->pdir, E_CHEB, use64, 1, h->q));
      RET(precond_gemvs(h, h->r, h->z, GH_CHEB_B, 1));
    } else {
      RET(launch_adat(h, h->pdir, E_PCG_A, use64, 1, h->q));
      RET(precond_gemvs(h, h->r, h->z, j + 1 == refine ? GH_PCG_B_LAST : GH_PCG_B, 1));
    }
  }
  RET(launch_adat(h, h->dy, E_TRUE_RES, true, 2, nullptr));
  RET(precond_gemvs(h, h->r, h->z, inner == LP_INNER_CHEBYSHEV ? GH_CHEB_REFRESH : GH_REFRESH, 2));
  return LP_OK;
}

// Whether the next block may be replayed from a graph: FP32 products, graphs
// enabled, and none of the block's products in the window opt.profile times
// (those blocks run as plain launches with events between them).
bool block_graph_usable(lp_handle* h, bool use64, int refine) {
  if (use64 || !h->opt.graphs || h->graphs_failed) return false;
  if (!h->opt.profile) return true;
  for (unsigned long long k = h->k1_sample; k < h->k1_sample + (unsigned long long)refine; ++k)
    if (((k >> 3) & 7) == 0) return false;
  return true;
}

// The block from its graph, captured on first use for this variant.  The
// packed d^2 the refresh reads is prepared outside the graph, so a replay
// never depends on what was valid at capture time.
int run_cg_block_graph(lp_handle* h, int inner, int refine) {
  if (!h->sparse && h->use_df && !h->d2df_valid) {
    DfPackArgs pk{{h->d2d}, {h->d2df}, 1, h->n};
    CK(launch_df_pack(pk, h->num_sms, h->st));
    h->d2df_valid = true;
  }
  const int key = refine * 8 + (h->qinv_ok ? 1 : 0) + (h->qinv_df_ok ? 2 : 0) + (h->opt.precondition ? 4 : 0);
  lp_handle::BlockGraph& g = h->blk_graph[inner == LP_INNER_CHEBYSHEV ? 1 : 0];
  if (!g.exec || g.key != key) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    const unsigned long long k1 = h->k1_sample;
    const long long before = g_launches.load();
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs_failed = true;
      return enqueue_cg_block(h, inner, false, refine);
    }
    const int rc = enqueue_cg_block(h, inner, false, refine);
    const cudaError_t ec = cudaStreamEndCapture(h->st, &graph);
    g.kernels = g_launches.load() - before;
    g_launches.fetch_sub(g.kernels, std::memory_order_relaxed);  // captured, not launched
    h->k1_sample = k1;
    cudaError_t ei = cudaErrorUnknown;
    if (rc == LP_OK && ec == cudaSuccess && graph)
      ei = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      g.exec = nullptr;
      h->graphs_failed = true;
      h->err.clear();
      return enqueue_cg_block(h, inner, false, refine);
    }
    g.key = key;
  }
  CK(cudaGraphLaunch(g.exec, h->st));
  g_launches.fetch_add(g.kernels, std::memory_order_relaxed);
  h->k1_sample += (unsigned long long)refine;
  h->graph_replays += 1;
  return LP_OK;
}

// The inner solve on the current factor: dy ~ M^{-1} p.  Returns LP_OK or
// LP_WARN_INNER_MAXIT (or kInnerSketchPoor when check_sketch is set).
// tol_f > 0: absolute ||f|| target; else relative tol_cg.
// warm: h->dy holds the starting point (CG only); otherwise dy^0 = 0 (Alg. 1)
int inner_solve(lp_handle* h, double tol_f, int* iters_out, bool warm = false,
                bool check_sketch = false, bool start64 = false) {
  const int m = h->m;
  int inner = h->opt.inner;
  if (warm && inner != LP_INNER_CG) warm = false;
  if (!warm) {
    CK(cudaMemsetAsync(h->dy, 0, sizeof(double) * m, h->st));
    CK(cudaMemcpyAsync(h->r, h->p, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  }
  CK(cudaMemsetAsync(&h->sc->inner_done, 0, 2 * sizeof(int), h->st));
  RET(set_scalar(h, &h->sc->tol_f, tol_f > 0 ? tol_f : 0.0));
  // r = p - M dy^0, unless the warm start just formed it from the same products
  if (warm && !h->warm_r_ready) RET(launch_adat(h, h->dy, E_TRUE_RES, true, 0, nullptr));
  h->warm_r_ready = false;
  const int refine = std::max(1, h->opt.refine_every);
  int total_iters = 0;
  if (inner == LP_INNER_CHEBYSHEV) {
    // interval from a few CG (Lanczos) steps on the same system
    RET(precond_gemvs(h, h->r, h->z, GH_PCG_INIT, 0));
    const int kl = std::max(2, h->opt.cheb_lanczos);
    RET(set_scalar(h, &h->sc->tol_f, 0.0));
    for (int j = 0; j < kl; ++j) {
      RET(launch_adat(h, h->pdir, E_PCG_A, false, 0, h->q));
      RET(precond_gemvs(h, h->r, h->z, GH_PCG_B, 0));
    }
    RET(sync_read(h));
    if (h->hsc->inner_done == 3) {
      *iters_out = total_iters + h->hsc->inner_iters;
      return kInnerIndefinite;
    }
    const int kk = std::min(kl, h->hsc->inner_iters);
    double tmin = 0.5, tmax = 2.0;
    RET(ritz_extremes(h, kk, &tmin, &tmax));
    total_iters += kk;
    // restart from dy = 0 with the Chebyshev recurrence
    CK(cudaMemsetAsync(h->dy, 0, sizeof(double) * m, h->st));
    CK(cudaMemcpyAsync(h->r, h->p, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemsetAsync(&h->sc->inner_done, 0, 2 * sizeof(int), h->st));
    RET(set_scalar(h, &h->sc->lam_min, 0.5 * tmin));
    RET(set_scalar(h, &h->sc->lam_max, 1.05 * tmax));
    RET(set_scalar(h, &h->sc->tol_f, tol_f > 0 ? tol_f : 0.0));
    RET(precond_gemvs(h, h->r, h->z, GH_CHEB_INIT, 0));
  } else {
    RET(precond_gemvs(h, h->r, h->z, GH_PCG_INIT, 0));
  }
  RET(sync_read(h));
  if (h->hsc->inner_done == 3) {
    *iters_out = total_iters;
    return kInnerIndefinite;
  }
  if (tol_f <= 0) {
    const double f0 = sqrt(std::max(h->hsc->rho0, 0.0));
    RET(set_scalar(h, &h->sc->tol_f, h->opt.tol_cg * f0));
    if (h->opt.tol_cg * f0 >= f0) {
      *iters_out = total_iters;
      return LP_OK;
    }
  } else if (h->hsc->inner_done == 2) {
    *iters_out = total_iters;
    return LP_OK;
  }
  int status = LP_OK;
  // FP32 products until a refresh shows the true residual stalled (the FP32
  // product's precision floor); then FP64 products for the rest of this solve.
  bool use64 = start64;
  double f_prev = h->hsc->f_true;
  // sketch check: Ritz values of the first refine-block of CG steps (one
  // unbroken Lanczos run from dy^0)
  check_sketch = check_sketch && inner == LP_INNER_CG && h->opt.precondition;
  bool poor = false, severe = false, ritz_done = false;
  while (true) {
    // refine steps, then the FP64 true residual r = p - M dy and
    // ||f|| = sqrt(r^T Q^{-1} r): replayed from a graph when it can be
    if (block_graph_usable(h, use64, refine)) RET(run_cg_block_graph(h, inner, refine));
    else RET(enqueue_cg_block(h, inner, use64, refine));
    CK(cudaMemcpyAsync(h->hsc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->hsc->err == ERR_NUMERICAL && !use64) {
      // A CG breakdown (p^T M p <= 0 or a non-finite value) with the FP32
      // product, on a matrix too ill-conditioned for it: the step that broke
      // was not applied, so continue from the current iterate with the
      // FP64-class product, restarting the recurrence from the true residual.
      use64 = true;
      h->breakdown_recoveries += 1;
      CK(cudaMemsetAsync(&h->sc->err, 0, sizeof(int), h->st));
      CK(cudaMemsetAsync(&h->sc->inner_done, 0, sizeof(int), h->st));
      RET(set_scalar(h, &h->sc->f_rec, 0.0));  // forces beta = 0 at the refresh
      if (inner == LP_INNER_CHEBYSHEV) inner = LP_INNER_CG;
      RET(launch_adat(h, h->dy, E_TRUE_RES, true, 0, nullptr));
      RET(precond_gemvs(h, h->r, h->z, GH_REFRESH, 0));
      RET(sync_read(h));
      f_prev = h->hsc->f_true;
      if (h->hsc->inner_done == 3) {
        status = kInnerIndefinite;
        break;
      }
      if (h->hsc->inner_done == 2) break;
      continue;
    }
    RET(check_read(h));  // the scalars were copied after the refresh just above
    if (h->opt.profile) ev_flush(h);
    if (h->hsc->inner_done == 3) {
      status = kInnerIndefinite;
      break;
    }
    if (h->hsc->inner_done == 2) break;
    if (h->hsc->inner_iters >= h->opt.t_max) {
      status = LP_WARN_INNER_MAXIT;
      break;
    }
    if (check_sketch && !ritz_done) {
      ritz_done = true;
      double lo = 0.0, hi = 0.0;
      RET(ritz_extremes(h, std::min(refine, h->hsc->inner_iters), &lo, &hi));
      poor = lo > 0.0 && hi > kRitzSpread * lo;
      severe = lo > 0.0 && hi > kRitzSevere * lo;
    }
    if (poor && (severe || h->hsc->inner_iters >= kPoorCheckIters)) {
      status = kInnerSketchPoor;
      break;
    }
    if (inner == LP_INNER_CHEBYSHEV && h->hsc->f_true > f_prev) {
      // The residual grew: the interval from the Lanczos estimate misses part
      // of the spectrum.  Continue with CG from the current iterate and the
      // refreshed residual (p = z, rho = r^T z).
      inner = LP_INNER_CG;
      RET(set_scalar(h, &h->sc->rho, h->hsc->f_true * h->hsc->f_true));
      CK(cudaMemcpyAsync(h->pdir, h->z, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
      h->cheb_fallbacks += 1;
    } else if (!use64 && h->hsc->f_true > 0.5 * f_prev) {
      use64 = true;
    }
    f_prev = h->hsc->f_true;
  }
  *iters_out = total_iters + h->hsc->inner_iters;
  return status;
}

// The sketch an inner solve runs on: D (or D^2), the outer index k and the
// retry index of the draw in use (updated when the draw is replaced).
struct SketchRef {
  const double* dvec;
  int is_d2;
  long long k;
  int* retry;
};

constexpr int kPoorRedraws = 4;
constexpr int kIndefRefactors = 2;

// inner_solve with three safeguards.
// (1) A draw of W that fails the embedding (kInnerSketchPoor) is replaced by the
//     next draw (retry + 1) and the solve continues from the current dy on the
//     new factor, at most kPoorRedraws times.
// (2) An indefinite stored Q^{-1} (kInnerIndefinite) is replaced by the FP64
//     Cholesky of the same Gram (sweep -> Cholesky) or the FP64 QR of (ADW)^T
//     (Cholesky -> QR), and the solve continues from the current dy.
//     In both cases the stopping rule keeps its target (relative targets are
//     re-based on the new factor's ||f(0)||).
// (3) Once more after refactoring by the QR of (ADW)^T when the iteration limit
//     was hit with the sweep's Q^{-1}: the sweep works on the Gram, which
//     squares kappa(ADW), and near degenerate vertices its double-float
//     accuracy can stop being enough for a useful preconditioner.
int inner_solve_robust(lp_handle* h, double tol_f, int* iters_out, bool warm = false,
                       const SketchRef* sk = nullptr) {
  int st = inner_solve(h, tol_f, iters_out, warm, sk != nullptr);
  int redraws = 0, refactors = 0;
  while (st == kInnerSketchPoor || st == kInnerIndefinite) {
    if (st == kInnerSketchPoor && (redraws >= kPoorRedraws || *sk->retry + 1 >= kMaxRetry)) {
      int more = 0;  // keep this draw: finish the solve without the check
      st = inner_solve(h, tol_f, &more, true, false);
      *iters_out += more;
      redraws = kPoorRedraws;
      continue;
    }
    if (st == kInnerSketchPoor) {
      redraws += 1;
      h->poor_redraws += 1;
      *sk->retry += 1;
      RET(sketch_and_factor(h, sk->dvec, sk->is_d2, sk->k, sk->retry));
    } else {
      if (h->factor_kind == 2 || refactors >= kIndefRefactors) {
        st = LP_WARN_INNER_MAXIT;  // no better factor to turn to
        break;
      }
      refactors += 1;
      h->indefinite_refactors += 1;
      const int rc = (h->factor_kind == 0 && h->blas) ? factor_chol(h) : factor_qr(h);
      const bool can_redraw = sk && redraws < kPoorRedraws && *sk->retry + 1 < kMaxRetry;
      const double ratio = h->hsc->diag_min > 0 ? h->hsc->diag_max / h->hsc->diag_min : INFINITY;
      if ((rc == LP_ERR_SKETCH_RANK || (rc == LP_OK && h->ratio_ref > 0.0 &&
                                         ratio > kRatioJump * h->ratio_ref)) && can_redraw) {
        // the FP64 factor shows the draw itself collapsed: replace it
        h->err.clear();
        redraws += 1;
        h->poor_redraws += 1;
        *sk->retry += 1;
        RET(sketch_and_factor(h, sk->dvec, sk->is_d2, sk->k, sk->retry));
      } else if (rc == LP_ERR_SKETCH_RANK) {
        // judged rank deficient in FP64: keep the solve so far on the sweep
        h->err.clear();
        RET(factor(h));
        st = LP_WARN_INNER_MAXIT;
        break;
      } else if (rc != LP_OK) {
        return rc;
      }
    }
    double tf = tol_f;
    if (tf <= 0) {  // relative rule: tol_cg ||f(0)|| in the new factor's norm
      RET(precond_gemvs(h, h->p, h->z, GH_NONE, 0));
      CK(launch_dot(h->m, h->p, h->z, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[1], h->num_sms, h->st));
      RET(sync_read(h));
      tf = h->opt.tol_cg * sqrt(std::max(h->hsc->pad[1], 0.0));
    }
    int more = 0;
    // after an indefinite Q^{-1} (kappa(Q)^2 u_DF >~ 1) the FP32 product's
    // error, about 2^-24 kappa(Q) in the preconditioned norm, is as large as
    // the operator: continue with the double-float product from the start
    st = inner_solve(h, tf, &more, true, sk != nullptr && redraws < kPoorRedraws, h->factor_kind != 0);
    *iters_out += more;
    tol_f = tf;
  }
  // a small t_max is the caller's choice, not a sign of a failed preconditioner
  if (st != LP_WARN_INNER_MAXIT || h->opt.t_max < 50 || !h->opt.precondition || !h->qinv_df_ok)
    return st;
  h->qr_refactors += 1;
  const int rc = factor_qr(h);
  if (rc == LP_ERR_SKETCH_RANK) {
    // the QR judges this sketch rank deficient: keep the first solve and restore
    // its factor (deterministic, so z = Q^{-1} r from the last refresh still holds)
    h->err.clear();
    RET(factor(h));
    return st;
  }
  if (rc != LP_OK) return rc;
  int more = 0;
  // the second attempt: FP64 factor of (ADW)^T and the double-float product
  st = inner_solve(h, tol_f, &more, false, false, true);
  *iters_out += more;
  return st == kInnerIndefinite ? LP_WARN_INNER_MAXIT : st;
}

// v = (XS)^{1/2} W (ADW)^T Q^{-1} (M dy - p); the last refresh left r = p - M dy
// and z = Q^{-1} r, so (ADW)^+ (M dy - p) = -(ADW)^T z.
int correction(lp_handle* h, const double* xs_x, const double* xs_s, long long k, int retry) {
  if (!h->opt.v_correction || !h->opt.precondition) {
    CK(cudaMemsetAsync(h->v, 0, sizeof(double) * h->npad, h->st));
    return LP_OK;
  }
  // One FP64 refinement step of z ~ Q^{-1} r with Q z = ADW (ADW^T z), so that
  // A S^{-1} v = A D^2 A^T dy - p (eq. addl) holds to FP64 accuracy whatever
  // the precision of the factor: e = r - Q z, z += R^{-1} R^{-T} e.
  CK(launch_adwt(h->adw, h->m, h->w, h->z, h->adwt_part, h->adwt_parts, h->uw, h->num_sms, h->st));
  CK(launch_gemv_rows(h->adw, h->m, h->w, h->uw, h->r, 1.0, -1.0, h->mb0, h->num_sms, h->st));
  if (h->qinv_ok) {
    CK(launch_gemv_tri(h->qinv, h->m, 2, h->mb0, h->z, GH_NONE, 0, nullptr, nullptr, nullptr, h->sc,
                       h->tickets + 1, &h->sc->err, 0, nullptr, h->num_sms, h->st, h->z,
                       h->qinv_df_ok ? h->qinv_df : nullptr));
  } else {
    CK(launch_gemv_tri(h->rinv_cm, h->m, 1, h->mb0, h->wv, GH_NONE, 0, nullptr, nullptr, nullptr,
                       h->sc, h->tickets + 1, &h->sc->err, 0, nullptr, h->num_sms, h->st));
    CK(launch_gemv_tri(h->rinv_rm, h->m, 0, h->wv, h->z, GH_NONE, 0, nullptr, nullptr, nullptr,
                       h->sc, h->tickets + 1, &h->sc->err, 0, nullptr, h->num_sms, h->st, h->z));
  }
  CK(launch_adwt(h->adw, h->m, h->w, h->z, h->adwt_part, h->adwt_parts, h->uw, h->num_sms, h->st));
  if (h->opt.sketch == LP_SKETCH_GAUSS)
    CK(launch_gauss_v(h->n, xs_x, xs_s, h->sk_dvec, h->sk_is_d2, h->uw, h->opt.seed, k, retry, h->w,
                      -1.0, h->v, h->num_sms, h->st));
  else
    CK(launch_v_gather(h->n, xs_x, xs_s, h->uw, h->opt.seed, k, retry, h->s_blocks, h->w, -1.0, h->v,
                       h->num_sms, h->st));
  return LP_OK;
}

// Warm start of the inner solve (fixed-sigma rule): features, recording, and a
// proposal.  The candidates v_1 = |u| model(X) (mode 2) and v_2 = dy_{k-1}
// (modes 1 and 2) are combined by one Galerkin step on M: dy^0 = sum c_i v_i
// with (v_i^T M v_j) c = (v_i^T p), the start of least energy-norm error
// ||M^{-1} p - dy^0||_M in their span, never worse than dy^0 = 0 in that norm.
// Its residual r^0 = p - sum c_i M v_i comes from the same products (one FP32
// product per candidate; the inner solve's first refresh replaces it by the
// FP64 residual), and dy^0 is used only when that residual beats dy^0 = 0.
// Leaves |u|^2 in sc->pad[0] for recording the target.
int warm_start_prepare(lp_handle* h, double mu_ratio, bool* warm) {
  *warm = false;
  h->warm_r_ready = false;
  if (h->ws_mode == 0 && !h->ws_rec_X) return LP_OK;
  const int m = h->m;
  RET(precond_gemvs(h, h->p, h->ws_u, GH_NONE, 0));  // u = Q^{-1} p
  CK(launch_dot(m, h->ws_u, h->ws_u, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[0], h->num_sms, h->st));
  CK(launch_dot(m, h->p, h->ws_u, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[1], h->num_sms, h->st));
  CK(launch_ws_features(m, h->dy_prev, h->ws_have_prev ? 1 : 0, h->ws_u, h->sc, h->ws_X, h->st));
  if (h->ws_rec_X && h->ws_count < h->ws_cap)
    CK(cudaMemcpyAsync(h->ws_rec_X + (size_t)h->ws_count * 3 * m, h->ws_X, sizeof(float) * 3 * m,
                       cudaMemcpyDeviceToDevice, h->st));
  const double* v[2];
  int nv = 0;
  if (h->ws_mode == 2 && h->ws_model) {
    if (mlp_predict(h->ws_model, h->ws_X, h->ws_hid, h->ws_Y, h->st) != LP_OK)
      return h->fail(LP_ERR_CUDA, "warm-start model forward failed");
    CK(launch_ws_scale(m, 0, h->ws_Y, nullptr, h->sc, h->ws_v, nullptr, h->st));
    v[nv++] = h->ws_v;
  }
  if (h->ws_mode != 0 && h->ws_have_prev) v[nv++] = h->dy_prev;
  // no proposals in the end game (mu < 1e-6 mu_0), where the iterates and the
  // preconditioner are most delicate and the inner solves are short anyway
  if (nv == 0 || h->opt.inner != LP_INNER_CG || mu_ratio < 1e-6) return LP_OK;
  h->ws_props += 1;
  const size_t wst = (size_t)h->lda + 64;
  double* wv[2] = {h->ws_w, h->ws_w + wst};
  // M v_i with the FP32 product: the coefficients need no more, and the first
  // refresh of the inner solve replaces r^0 by the FP64 residual
  for (int i = 0; i < nv; ++i) RET(launch_adat(h, v[i], E_PLAIN, false, 0, wv[i]));
  // dots: [0] v0.Mv0 [1] v0.Mv1 [2] v1.Mv0 [3] v1.Mv1 [4] v0.p [5] v1.p
  for (int i = 0; i < nv; ++i) {
    for (int j = 0; j < nv; ++j)
      CK(launch_dot(m, v[i], wv[j], 1.0, h->vpart, h->tickets + 3, h->ws_dots + 2 * i + j, h->num_sms, h->st));
    CK(launch_dot(m, v[i], h->p, 1.0, h->vpart, h->tickets + 3, h->ws_dots + 4 + i, h->num_sms, h->st));
  }
  double g[6] = {0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(g, h->ws_dots, sizeof g, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  double c0 = 0.0, c1 = 0.0;
  const double g01 = 0.5 * (g[1] + g[2]);
  const double det = g[0] * g[3] - g01 * g01;
  if (nv == 2 && g[0] > 0.0 && g[3] > 0.0 && det > 1e-10 * g[0] * g[3]) {
    c0 = (g[4] * g[3] - g01 * g[5]) / det;
    c1 = (g[0] * g[5] - g01 * g[4]) / det;
  } else if (g[0] > 0.0) {
    c0 = g[4] / g[0];  // the first candidate alone
    nv = 1;
  } else {
    return LP_OK;
  }
  CK(launch_axpby(m, c0, v[0], nv == 2 ? c1 : 0.0, nv == 2 ? v[1] : v[0], h->dy, h->num_sms, h->st));
  CK(launch_axpby(m, 1.0, h->p, -c0, wv[0], h->r, h->num_sms, h->st));  // r^0 = p - sum c_i M v_i
  if (nv == 2) CK(launch_axpby(m, 1.0, h->r, -c1, wv[1], h->r, h->num_sms, h->st));
  RET(precond_gemvs(h, h->r, h->z, GH_NONE, 0));
  CK(launch_dot(m, h->r, h->z, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[2], h->num_sms, h->st));
  CK(launch_dot(m, h->dy, h->dy, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[3], h->num_sms, h->st));
  RET(sync_read(h));
  // ||f(dy^0)|| < ||f(0)|| (Q^{-1}-norms), and no large component along nearly
  // null directions of M, which the residual does not see but which would raise
  // the rounding floor of the refreshed residual: |dy^0| <= 4 |Q^{-1} p|
  // (Q^{-1} p approximates dy = M^{-1} p within the preconditioner's spread)
  if (h->hsc->pad[2] < h->hsc->pad[1] && h->hsc->pad[3] <= 16.0 * h->hsc->pad[0]) {
    *warm = true;
    h->warm_r_ready = true;
    h->ws_acc += 1;
  }
  return LP_OK;
}

// after the inner solve: record the target, keep dy for the next proposal
int warm_start_finish(lp_handle* h) {
  const int m = h->m;
  if (h->ws_rec_X && h->ws_count < h->ws_cap) {
    CK(launch_ws_scale(m, 1, nullptr, h->dy, h->sc, nullptr, h->ws_rec_T + (size_t)h->ws_count * m, h->st));
    h->ws_count += 1;
  }
  if (h->ws_mode != 0 || h->ws_rec_X) {
    CK(cudaMemcpyAsync(h->dy_prev, h->dy, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
    h->ws_have_prev = true;
  }
  return LP_OK;
}

int copy_in(lp_handle* h, double* dst, const double* src, size_t count, int on_device) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * count,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  return LP_OK;
}

int copy_out(lp_handle* h, double* dst, const double* src, size_t count, int on_device) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * count,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  return LP_OK;
}

int residual_pass(lp_handle* h, bool feasible, double sigma = -1.0) {
  StreamArgs a = base_args(h);
  a.feasible = feasible ? 1 : 0;
  if (sigma >= 0.0) a.sigma = sigma;
  a.cv[0] = h->x;
  a.cv[1] = h->s;
  a.cv[2] = h->c;
  a.cv_esz[0] = a.cv_esz[1] = a.cv_esz[2] = 8;
  a.ncv = 3;
  a.vin = h->y;
  a.out_col[0] = h->rd;
  a.out_col[1] = h->d2d;
  a.out_colf = h->d2f;
  a.red_partials = h->red_partials;
  a.epilogue = E_RESID;
  a.out_m0 = h->rp;
  a.out_m1 = h->p;
  a.bvec = h->b;
  if (!h->sparse && h->use_df_resid) {
    // double-float pass: x, s (and the constant c) as pairs in, r_d and d2 as pairs out
    DfPackArgs pk{{h->x, h->s}, {h->dfin[0], h->dfin[1]}, 2, h->n};
    CK(launch_df_pack(pk, h->num_sms, h->st));
    a.cv[0] = h->dfin[0];
    a.cv[1] = h->dfin[1];
    a.cv[2] = h->cdf;
    a.out_df[0] = h->dfout[0];
    a.out_df[1] = h->d2df;
    a.red_partials = nullptr;
    if (h->use_rows) CK(launch_rows(h->dtype, true, M_RESID, a, h->rplan_df, h->st, false));
    else CK(launch_stream_df(h->dtype, M_RESID, a, h->plan, h->st));
    DfUnpackArgs up{0, h->n, h->dfout[0], h->d2df, h->rd, h->d2d, h->d2f, h->x, h->s, h->c, h->sc,
                    h->vpart, h->tickets + 7};
    CK(launch_df_unpack(up, h->num_sms, h->st));
    h->d2df_valid = true;
    return LP_OK;
  }
  h->d2df_valid = false;
  if (h->sparse) CK(launch_sparse2(h->dtype, true, M_RESID, a, h->num_sms, h->st));
  else CK(launch_stream(h->dtype, true, M_RESID, a, h->plan, h->st));
  return LP_OK;
}

int direction_pass(lp_handle* h, bool feasible, double sigma = -1.0) {
  StreamArgs a = base_args(h);
  a.feasible = feasible ? 1 : 0;
  if (sigma >= 0.0) a.sigma = sigma;
  a.cv[0] = h->x;
  a.cv[1] = h->s;
  a.cv[2] = h->v;
  a.cv[3] = h->rd;
  a.cv_esz[0] = a.cv_esz[1] = a.cv_esz[2] = a.cv_esz[3] = 8;
  a.ncv = feasible ? 3 : 4;
  a.vin = h->dy;
  a.out_col[0] = h->dx;
  a.out_col[1] = h->ds;
  a.red_partials = h->red_partials;
  a.epilogue = E_DIR;
  if (h->sparse) CK(launch_sparse2(h->dtype, true, M_DIR, a, h->num_sms, h->st));
  else if (h->use_df_dir) {
    // double-float pass: x, s, v, r_d as pairs in, dx and ds as pairs out
    DfPackArgs pk{{h->x, h->s, h->v, h->rd}, {h->dfin[0], h->dfin[1], h->dfin[2], h->dfin[3]},
                  feasible ? 3 : 4, h->n};
    CK(launch_df_pack(pk, h->num_sms, h->st));
    for (int q = 0; q < 4; ++q) {
      a.cv[q] = h->dfin[q];
      a.cv_esz[q] = 8;
    }
    a.ncv = feasible ? 3 : 4;
    a.out_df[0] = h->dfout[0];
    a.out_df[1] = h->dfout[1];
    a.red_partials = nullptr;
    if (h->use_rows) CK(launch_rows(h->dtype, true, M_DIR, a, h->rplan_df, h->st, false));
    else CK(launch_stream_df(h->dtype, M_DIR, a, h->plan, h->st));
    DfUnpackArgs up{1, h->n, h->dfout[0], h->dfout[1], h->dx, h->ds, nullptr, h->x, h->s, nullptr, h->sc,
                    h->vpart, h->tickets + 7};
    CK(launch_df_unpack(up, h->num_sms, h->st));
  }
  else CK(launch_stream(h->dtype, true, M_DIR, a, h->plan, h->st));
  return LP_OK;
}

int compute_mu(lp_handle* h) {
  CK(launch_dot(h->n, h->x, h->s, 1.0 / (double)h->n, h->vpart, h->tickets + 3, &h->sc->mu,
                h->num_sms, h->st));
  return LP_OK;
}

void options_check(const lp_options* o, std::string* why) {
  if (!(o->sigma > 0 && o->sigma < 1)) *why = "sigma must be in (0, 1)";
  else if (!(o->gamma > 0 && o->gamma < 1)) *why = "gamma must be in (0, 1)";
  else if (o->s < 1 || o->s > kMaxBlocks) *why = "s must be in [1, 16]";
  else if (o->sketch != LP_SKETCH_COUNT && o->sketch != LP_SKETCH_GAUSS) *why = "unknown sketch";
  else if (o->precondition != 0 && o->precondition != 1) *why = "precondition must be 0 or 1";
  else if (o->sigma_rule != 0 && o->sigma_rule != 1) *why = "sigma_rule must be 0 or 1";
  else if (o->inner != LP_INNER_CG && o->inner != LP_INNER_CHEBYSHEV) *why = "inner must be CG or Chebyshev";
  else if (o->t_max < 1 || o->k_max < 0) *why = "t_max >= 1 and k_max >= 0 required";
  else if (o->inner_rule != LP_RULE_THEORY && o->inner_rule != LP_RULE_RELATIVE) *why = "unknown inner_rule";
  else if (!(o->tol_cg >= 0 && std::isfinite(o->tol_cg))) *why = "tol_cg must be finite and >= 0";
  else if (o->w < 0) *why = "w must be >= 0 (0: w = w_factor m)";
  else if (o->w == 0 && !(o->w_factor > 0 && o->w_factor <= 1e6)) *why = "w_factor must be in (0, 1e6] when w = 0";
  else if (o->graphs != 0 && o->graphs != 1) *why = "graphs must be 0 or 1";
  else if (o->autotune != 0 && o->autotune != 1) *why = "autotune must be 0 or 1";
  else if (o->guard != 0 && o->guard != 1) *why = "guard must be 0 or 1";
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {
// C++ exceptions must not cross the C ABI: each entry point that allocates on
// the host maps one to a status code (bad_alloc: LP_ERR_OOM; a size the
// standard library refuses: LP_ERR_ARG) and records a message.
template <typename F>
int guarded(std::string* err, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    if (err) *err = "host allocation failed";
    return LP_ERR_OOM;
  } catch (const std::exception& e) {
    if (err) *err = std::string("invalid size: ") + e.what();
    return LP_ERR_ARG;
  } catch (...) {
    if (err) *err = "unexpected host exception";
    return LP_ERR_ARG;
  }
}
}  // namespace

extern "C" {

void lp_options_default(lp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->sigma = 0.5;
  o->gamma = 0.999;
  o->tol_cg = 1e-5;
  o->inner_rule = LP_RULE_THEORY;
  o->sketch = LP_SKETCH_COUNT;
  o->s = 2;
  o->inner = LP_INNER_CG;
  o->refine_every = 8;
  o->k_max = 200;
  o->t_max = 500;
  o->v_correction = 1;
  o->cheb_lanczos = 10;
  o->profile = 0;
  o->w_factor = 4.0;
  o->w = 0;
  o->seed = 0;
  o->stream = nullptr;
  o->tensor_sketch = 1;
  o->precondition = 1;
  o->sigma_rule = 0;
  o->graphs = 1;
  o->autotune = 0;
  o->guard = 0;
}

const char* lp_create_error(void) { return g_create_error.c_str(); }

const char* lp_last_error(const lp_handle* h) { return h ? h->err.c_str() : ""; }

int lp_destroy(lp_handle* h) {
  if (!h) return LP_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto& e : h->ev_pool) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (h->st_aux) cudaStreamSynchronize(h->st_aux);  // no kernel of this handle uses a block any more
  for (auto& a : h->allocs) pool_give(h->dev, a.second, a.first);
  if (h->hsc) cudaFreeHost(h->hsc);
  if (h->hinfo) cudaFreeHost(h->hinfo);
  if (h->hval) cudaFreeHost(h->hval);
  if (h->hwork) free(h->hwork);
  for (auto& g : h->blk_graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->sol) cusolverDnDestroy(h->sol);
  if (h->blas) cublasDestroy(h->blas);
  if (h->st_aux) {
    cudaStreamSynchronize(h->st_aux);
    cudaStreamDestroy(h->st_aux);
  }
  if (h->ev_x) cudaEventDestroy(h->ev_x);
  if (h->ev_p) cudaEventDestroy(h->ev_p);
  if (h->ev_cor) cudaEventDestroy(h->ev_cor);
  if (h->ev_step) cudaEventDestroy(h->ev_step);
  if (h->ev_end) cudaEventDestroy(h->ev_end);
  if (h->ev_res) cudaEventDestroy(h->ev_res);
  if (h->ev_res_end) cudaEventDestroy(h->ev_res_end);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
  return LP_OK;
}

// ---------------------------------------------------------------------------
// autotuner of the inner-loop product's tile shape (opt.autotune)
// ---------------------------------------------------------------------------
// Candidates for the FP32 product A diag(d2) A^T v on this handle's A: the
// warp-per-column kernel with tiles of about 16, 32 or 64 KB and 2 to 4
// stages, and the row-split kernel where the rows allow; each runs once
// untimed and three times between CUDA events on the handle's stream, and the
// fastest is kept for the handle and cached for the process, keyed by the
// storage dtype, the leading dimension and n, so that every later handle of
// the same shape takes the same kernel without timing (results then agree
// bit for bit between handles; a different choice changes the summation
// order, so autotuned results agree with untuned ones to rounding).
namespace {
struct TuneKey {
  int dtype, lda;
  long long n;
  bool operator<(const TuneKey& o) const {
    return dtype != o.dtype ? dtype < o.dtype : (lda != o.lda ? lda < o.lda : n < o.n);
  }
};
struct TuneChoice {
  bool rows = false;
  int target = 0, stages = 0;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneChoice> g_tune_cache;
}  // namespace

static void apply_choice(lp_handle* h, const TuneChoice& c) {
  h->prod_rows = c.rows;
  if (!c.rows) h->fplan = make_stream_plan_ex(h->m, h->n, h->lda, h->esz, h->num_sms, 4, c.target, c.stages);
}

static int autotune_product(lp_handle* h) {
  const TuneKey key{h->dtype, h->lda, h->n};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply_choice(h, it->second);
      return LP_OK;
    }
  }
  std::vector<TuneChoice> cand;
  const int vpl = fused_vpl(h->lda, h->esz);
  if (vpl >= 1 && vpl <= 8)
    for (int target : {16 * 1024, 32 * 1024, 64 * 1024})
      for (int stages : {2, 3, 4}) {
        const StreamPlan p = make_stream_plan_ex(h->m, h->n, h->lda, h->esz, h->num_sms, 4, target, stages);
        if (p.ok && p.stages == stages && p.grid <= h->alloc_grid) cand.push_back(TuneChoice{false, target, stages});
      }
  if (h->rplan.ok && h->rplan.grid <= h->alloc_grid) cand.push_back(TuneChoice{true, 0, 0});
  if (cand.empty()) return LP_OK;
  // d2 = 1, v = 1 in the handle's work vectors
  CK(launch_fill(h->n, h->d2d, 1.0, h->num_sms, h->st));
  CK(launch_to_f32(h->n, h->d2d, h->d2f, 0, h->num_sms, h->st));
  h->d2df_valid = false;
  CK(launch_fill(h->m, h->mb0, 1.0, h->num_sms, h->st));
  CK(cudaMemsetAsync(&h->sc->inner_done, 0, 2 * sizeof(int), h->st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return h->fail(LP_ERR_CUDA, "cudaEventCreate failed");
  }
  const int profile = h->opt.profile;
  h->opt.profile = 0;  // no sampled events while timing candidates
  float best = 0.0f;
  int best_i = -1, rc = LP_OK;
  for (size_t i = 0; i < cand.size() && rc == LP_OK; ++i) {
    apply_choice(h, cand[i]);
    rc = launch_adat(h, h->mb0, E_PLAIN, false, 0, h->mb1);
    if (rc != LP_OK) break;
    cudaEventRecord(e0, h->st);
    for (int r = 0; r < 3 && rc == LP_OK; ++r) rc = launch_adat(h, h->mb0, E_PLAIN, false, 0, h->mb1);
    cudaEventRecord(e1, h->st);
    float ms = 0.0f;
    if (rc == LP_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        (best_i < 0 || ms < best)) {
      best = ms;
      best_i = (int)i;
    }
  }
  h->opt.profile = profile;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LP_OK) return rc;
  RET(sync_read(h));
  if (best_i < 0) return h->fail(LP_ERR_CUDA, "autotune: no candidate could be timed");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto ins = g_tune_cache.emplace(key, cand[best_i]);
    apply_choice(h, ins.first->second);  // a concurrent tuner may have cached first: take its choice
  }
  return LP_OK;
}

// The sparse A by rows for the two-pass kernels: CSR from the CSC (the same
// stable counting sort, read as CSC of A = CSR of A^T), rows split into
// segments of at most kSegNnz entries, and the per-column scalars and
// segment sums the passes exchange.  A device CSC is read back first.
static int build_rows(lp_handle* h, const lp_matrix* A) {
  const int esz = h->esz;
  const long long nnz = h->nnz, n = h->n;
  const int m = h->m;
  std::vector<int64_t> cp_h;
  std::vector<int32_t> ri_h;
  std::vector<char> v_h;
  const int64_t* cp = A->ptr;
  const int32_t* ri = A->idx;
  const void* vv = A->val;
  if (A->on_device) {
    cp_h.resize((size_t)n + 1);
    ri_h.resize((size_t)std::max<long long>(nnz, 1));
    v_h.resize((size_t)std::max<long long>(nnz, 1) * esz);
    CK(cudaMemcpy(cp_h.data(), A->ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost));
    if (nnz > 0) {
      CK(cudaMemcpy(ri_h.data(), A->idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(v_h.data(), A->val, (size_t)esz * nnz, cudaMemcpyDeviceToHost));
    }
    cp = cp_h.data();
    ri = ri_h.data();
    vv = v_h.data();
  }
  if (n > INT32_MAX) return h->fail(LP_ERR_UNSUPPORTED, "sparse n too large for the row form");
  CscCopy rows;  // CSC of A^T = CSR of A
  const std::string bad = csr_to_csc((int)n, m, nnz, cp, ri, vv, esz, &rows);
  if (!bad.empty()) return h->fail(LP_ERR_ARG, "CSC structure: %s", bad.c_str());
  // segments
  std::vector<long long> seg;
  std::vector<int> seg_row, row_seg((size_t)m + 1, 0);
  for (int i = 0; i < m; ++i) {
    row_seg[i] = (int)seg_row.size();
    for (long long k = rows.ptr[i]; k < rows.ptr[i + 1]; k += kSegNnz) {
      seg.push_back(k);
      seg.push_back(std::min<long long>(rows.ptr[i + 1], k + kSegNnz));
      seg_row.push_back(i);
    }
  }
  row_seg[m] = (int)seg_row.size();
  h->nseg = (int)seg_row.size();
  RET(h->alloc(&h->rowptr, (size_t)m + 1));
  RET(h->alloc(&h->colidx, (size_t)std::max<long long>(nnz, 1)));
  RET(h->alloc(reinterpret_cast<char**>(&h->rval), (size_t)std::max<long long>(nnz, 1) * esz));
  RET(h->alloc(&h->seg, 2 * (size_t)std::max(h->nseg, 1)));
  RET(h->alloc(&h->seg_row, (size_t)std::max(h->nseg, 1)));
  RET(h->alloc(&h->row_seg, (size_t)m + 1));
  RET(h->alloc(&h->tcol, 2 * (size_t)h->npad));
  RET(h->alloc(&h->segsum, 2 * (size_t)std::max(h->nseg, 1) + 2 + 2 * (size_t)sparse2_col_grid(n, h->num_sms)));
  CK(cudaMemcpyAsync(h->rowptr, rows.ptr.data(), sizeof(int64_t) * ((size_t)m + 1), cudaMemcpyHostToDevice, h->st));
  if (nnz > 0) {
    CK(cudaMemcpyAsync(h->colidx, rows.idx.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->rval, rows.val.data(), (size_t)esz * nnz, cudaMemcpyHostToDevice, h->st));
  }
  if (h->nseg > 0) {
    CK(cudaMemcpyAsync(h->seg, seg.data(), sizeof(long long) * seg.size(), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->seg_row, seg_row.data(), sizeof(int) * seg_row.size(), cudaMemcpyHostToDevice, h->st));
  }
  CK(cudaMemcpyAsync(h->row_seg, row_seg.data(), sizeof(int) * row_seg.size(), cudaMemcpyHostToDevice, h->st));
  // the host vectors go out of scope: wait for the copies from them
  CK(cudaStreamSynchronize(h->st));
  return LP_OK;
}

static int create_impl(lp_handle* h, const lp_matrix* A, const double* b, const double* c,
                       int bc_on_device, const lp_options* opt) {
  if (!A || !b || !c) return h->fail(LP_ERR_ARG, "A, b and c are required");
  if (A->m < 1 || A->n < A->m) return h->fail(LP_ERR_ARG, "need 1 <= m <= n (m=%d n=%lld)", A->m, (long long)A->n);
  if (A->fmt != LP_DENSE_COLMAJOR && A->fmt != LP_CSC && A->fmt != LP_CSR)
    return h->fail(LP_ERR_ARG, "bad format");
  if (A->dtype < LP_F64 || A->dtype > LP_BF16) return h->fail(LP_ERR_ARG, "bad dtype");
  if (A->fmt == LP_DENSE_COLMAJOR && (!A->val || A->ld < A->m))
    return h->fail(LP_ERR_ARG, "dense A needs val and ld >= m");
  if (A->fmt == LP_CSR) {
    if (!A->val || !A->ptr || !A->idx || A->nnz < 0) return h->fail(LP_ERR_ARG, "CSR A needs ptr, idx, val");
    if (A->dtype == LP_BF16) return h->fail(LP_ERR_UNSUPPORTED, "CSR values must be FP32 or FP64");
    if (A->nnz >= (1LL << 40)) return h->fail(LP_ERR_ARG, "nnz too large");
    if (A->n > INT32_MAX) return h->fail(LP_ERR_ARG, "CSR column indices are 32-bit: n too large");
  }
  if (A->fmt == LP_CSC) {
    if (!A->val || !A->ptr || !A->idx || A->nnz < 0) return h->fail(LP_ERR_ARG, "CSC A needs ptr, idx, val");
    if (A->dtype == LP_BF16) return h->fail(LP_ERR_UNSUPPORTED, "CSC values must be FP32 or FP64");
    if (A->nnz >= (1LL << 40)) return h->fail(LP_ERR_ARG, "nnz too large");
    if (!A->on_device) {  // structural check of a host CSC
      if (A->ptr[0] != 0 || A->ptr[A->n] != A->nnz) return h->fail(LP_ERR_ARG, "CSC ptr[0] != 0 or ptr[n] != nnz");
      for (long long j = 0; j < A->n; ++j)
        if (A->ptr[j + 1] < A->ptr[j]) return h->fail(LP_ERR_ARG, "CSC ptr not monotone");
      for (long long q = 0; q < A->nnz; ++q)
        if (A->idx[q] < 0 || A->idx[q] >= A->m) return h->fail(LP_ERR_ARG, "CSC row index out of range");
    }
  }
  lp_options_default(&h->opt);
  if (opt) h->opt = *opt;
  std::string why;
  options_check(&h->opt, &why);
  if (!why.empty()) return h->fail(LP_ERR_ARG, "%s", why.c_str());
  // sketch width (host data only: every argument error is found before the
  // first CUDA call)
  h->s_blocks = h->opt.s;
  long long w = h->opt.w > 0 ? h->opt.w : (long long)llround(h->opt.w_factor * A->m);
  w = round_up_ll(std::max<long long>(w, h->s_blocks), h->s_blocks);
  if (w < A->m) return h->fail(LP_ERR_ARG, "sketch width w=%lld < m=%d: A D W cannot have rank m", w, A->m);
  if (w > (1 << 30)) return h->fail(LP_ERR_ARG, "sketch width too large");
  h->w = (int)w;
  if (A->fmt != LP_DENSE_COLMAJOR && h->opt.sketch == LP_SKETCH_GAUSS)
    return h->fail(LP_ERR_UNSUPPORTED, "the Gaussian sketch is built for dense A only");
  // CSR input: the sparse kernels stream columns, so the rows are sorted into
  // CSC here (a device CSR is read back to the host first)
  lp_matrix csc_view;
  CscCopy conv;
  if (A->fmt == LP_CSR) {
    const int esz_in = A->dtype == LP_F64 ? 8 : 4;
    const int64_t* rp = A->ptr;
    const int32_t* ci = A->idx;
    const void* vv = A->val;
    std::vector<int64_t> rp_h;
    std::vector<int32_t> ci_h;
    std::vector<char> vv_h;
    if (A->on_device) {
      rp_h.resize((size_t)A->m + 1);
      ci_h.resize((size_t)std::max<long long>(A->nnz, 1));
      vv_h.resize((size_t)std::max<long long>(A->nnz, 1) * esz_in);
      CK(cudaMemcpy(rp_h.data(), A->ptr, sizeof(int64_t) * ((size_t)A->m + 1), cudaMemcpyDeviceToHost));
      if (A->nnz > 0) {
        CK(cudaMemcpy(ci_h.data(), A->idx, sizeof(int32_t) * (size_t)A->nnz, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(vv_h.data(), A->val, (size_t)esz_in * A->nnz, cudaMemcpyDeviceToHost));
      }
      rp = rp_h.data();
      ci = ci_h.data();
      vv = vv_h.data();
    }
    const std::string bad = csr_to_csc(A->m, A->n, A->nnz, rp, ci, vv, esz_in, &conv);
    if (!bad.empty()) return h->fail(LP_ERR_ARG, "%s", bad.c_str());
    csc_view = *A;
    csc_view.fmt = LP_CSC;
    csc_view.ptr = conv.ptr.data();
    csc_view.idx = conv.idx.data();
    csc_view.val = conv.val.data();
    csc_view.on_device = 0;
    A = &csc_view;
  }
  CK(cudaGetDevice(&h->dev));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev));
  if (h->opt.stream) {
    h->st = static_cast<cudaStream_t>(h->opt.stream);
  } else {
    CK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CK(cudaStreamCreateWithFlags(&h->st_aux, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_x, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_p, cudaEventDisableTiming));
  CK(cudaEventCreate(&h->ev_cor));
  CK(cudaEventCreate(&h->ev_step));
  CK(cudaEventCreate(&h->ev_end));
  CK(cudaEventCreate(&h->ev_res));
  CK(cudaEventCreate(&h->ev_res_end));
  h->m = A->m;
  h->n = A->n;
  h->dtype = A->dtype;
  h->fmt = A->fmt;
  h->esz = A->dtype == LP_F64 ? 8 : (A->dtype == LP_F32 ? 4 : 2);
  const int vec = 16 / h->esz;
  h->lda = (int)round_up_ll(h->m, vec);
  h->npad = round_up_ll(h->n, 64);
  h->sparse = A->fmt == LP_CSC;
  if (h->sparse) {
    h->lda = (int)round_up_ll(h->m, 4);
    if (h->lda * 3 * 8 > 200 * 1024)
      return h->fail(LP_ERR_UNSUPPORTED, "m=%d too large for the CSC kernels' shared-memory vectors", h->m);
    h->sp_grid = sparse_grid(h->num_sms);
    h->plan.grid = h->sp_grid;
    h->plan.ok = true;
  }
  // kernel shape limits
  if (!h->sparse) h->plan = make_stream_plan(h->m, h->n, h->lda, h->esz, h->num_sms, 4);
  h->use_df = !h->sparse && h->dtype != LP_F64 && stream_df_supported(M_ADAT, h->lda, h->esz, h->plan);
  h->use_df_resid = !h->sparse && h->dtype != LP_F64 && stream_df_supported(M_RESID, h->lda, h->esz, h->plan);
  h->use_df_dir = !h->sparse && h->dtype != LP_F64 && stream_df_supported(M_DIR, h->lda, h->esz, h->plan);
  // Tall columns (16-byte vectors per lane per column >= 8: m > 512 in FP32,
  // m > 1024 in BF16) go to the row-split kernels, whose per-lane state does
  // not grow with m; the warp-per-column kernels would spill there.
  if (!h->sparse && h->dtype != LP_F64) {
    const int vpl = fused_vpl(h->lda, h->esz);
    h->rplan = make_rows_plan(h->lda, h->n, h->esz, h->num_sms, false);
    h->rplan_df = make_rows_plan(h->lda, h->n, h->esz, h->num_sms, true);
    h->use_rows = h->rplan.ok && h->rplan_df.ok && (vpl == 0 || vpl >= 8);
    if (h->use_rows) h->use_df = h->use_df_resid = h->use_df_dir = true;
    h->prod_rows = h->use_rows;
    h->fplan = h->plan;
  }
  if (!h->plan.ok) return h->fail(LP_ERR_UNSUPPORTED, "m=%d too large for the streaming kernels", h->m);
  if (!h->sparse && h->dtype != LP_F64 && fused_vpl(h->lda, h->esz) == 0 && !h->use_rows)
    return h->fail(LP_ERR_UNSUPPORTED, "m=%d too large for the fused product kernel", h->m);
  if (!h->sparse && h->lda / vec > 4 * kThreads)
    return h->fail(LP_ERR_UNSUPPORTED, "m=%d too large for the FP64 streaming kernel", h->m);
  // device memory
  const size_t n = (size_t)h->npad, m = (size_t)h->lda;
  const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (h->sparse) {
    h->nnz = A->nnz;
    RET(h->alloc(&h->colptr, (size_t)h->n + 1));
    RET(h->alloc(&h->rowidx, (size_t)std::max<long long>(h->nnz, 1)));
    RET(h->alloc(reinterpret_cast<char**>(&h->spval), (size_t)std::max<long long>(h->nnz, 1) * h->esz));
    CK(cudaMemcpyAsync(h->colptr, A->ptr, sizeof(long long) * ((size_t)h->n + 1), kind, h->st));
    if (h->nnz > 0) {
      CK(cudaMemcpyAsync(h->rowidx, A->idx, sizeof(int) * (size_t)h->nnz, kind, h->st));
      CK(cudaMemcpyAsync(h->spval, A->val, (size_t)h->esz * h->nnz, kind, h->st));
    }
    RET(build_rows(h, A));
    // the bucket lists of the reproducible sparse CountSketch (else FP64 atomics)
    if (h->opt.sketch == LP_SKETCH_COUNT && h->w <= kCsMaxW && (long long)h->n * h->s_blocks < (1LL << 31) &&
        h->m <= kSpMaxRows) {
      RET(h->alloc(&h->cs.count, (size_t)h->w + 1));
      RET(h->alloc(&h->cs.base, (size_t)h->w + 1));
      RET(h->alloc(&h->cs.cursor, (size_t)h->w + 1));
      RET(h->alloc(&h->cs.list, (size_t)h->n * h->s_blocks));
      RET(h->alloc(&h->cs.sc64, (size_t)h->n));
      RET(h->alloc(&h->cs.scdf, (size_t)h->n));
    }
  } else {
    if (h->opt.sketch == LP_SKETCH_COUNT) {
      if (h->w > kCsMaxW)
        return h->fail(LP_ERR_UNSUPPORTED, "sketch width w=%d above %d for the dense CountSketch", h->w, kCsMaxW);
      if ((long long)h->n * h->s_blocks >= (1LL << 31))
        return h->fail(LP_ERR_UNSUPPORTED, "n * s too large for the CountSketch bucket lists");
      RET(h->alloc(&h->cs.count, (size_t)h->w + 1));
      RET(h->alloc(&h->cs.base, (size_t)h->w + 1));
      RET(h->alloc(&h->cs.cursor, (size_t)h->w + 1));
      RET(h->alloc(&h->cs.list, (size_t)h->n * h->s_blocks));
      RET(h->alloc(&h->cs.sc64, (size_t)h->n));
      RET(h->alloc(&h->cs.scdf, (size_t)h->n));
    }
    RET(h->alloc(reinterpret_cast<char**>(&h->A), (size_t)h->lda * h->n * h->esz));
    if (A->ld == h->lda && h->m == h->lda) {
      // no padding on either side: one contiguous copy (a pitched copy of n
      // short rows moves the same bytes several times slower)
      CK(cudaMemcpyAsync(h->A, A->val, (size_t)h->lda * h->n * h->esz, kind, h->st));
    } else {
      CK(cudaMemcpy2DAsync(h->A, (size_t)h->lda * h->esz, A->val, (size_t)A->ld * h->esz,
                           (size_t)h->m * h->esz, (size_t)h->n, kind, h->st));
    }
  }
  double** nvecs[] = {&h->c, &h->x, &h->y, &h->s, &h->rd, &h->d2d, &h->dx, &h->ds, &h->v,
                      &h->nb0, &h->nb1, &h->nb2};
  for (double** p : nvecs) RET(h->alloc(p, n));
  RET(h->alloc(&h->d2f, n));
  if (!h->sparse && h->dtype != LP_F64) {
    for (int q = 0; q < 4; ++q) RET(h->alloc(&h->dfin[q], n));
    for (int q = 0; q < 2; ++q) RET(h->alloc(&h->dfout[q], n));
    RET(h->alloc(&h->d2df, n));
    RET(h->alloc(&h->cdf, n));
  }
  double** mvecs[] = {&h->b, &h->rp, &h->p, &h->dy, &h->r, &h->z, &h->pdir, &h->q, &h->wv,
                      &h->mb0, &h->mb1};
  for (double** p : mvecs) RET(h->alloc(p, m + 64));
  RET(h->alloc(&h->coef, std::max<size_t>(2 * (size_t)h->opt.t_max, 2048) + 64));
  CK(cudaMemcpyAsync(h->b, b, sizeof(double) * h->m,
                     bc_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->c, c, sizeof(double) * h->n,
                     bc_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  if (h->cdf) {
    DfPackArgs pk{{h->c}, {h->cdf}, 1, h->n};
    CK(launch_df_pack(pk, h->num_sms, h->st));
  }
  const size_t mw = (size_t)h->m * h->w;
  RET(h->alloc(&h->adw, mw));
  RET(h->alloc(&h->qr, mw));
  RET(h->alloc(&h->tau, (size_t)h->m));
  RET(h->alloc(&h->rinv_cm, (size_t)h->m * h->m));
  RET(h->alloc(&h->rinv_rm, (size_t)h->m * h->m));
  RET(h->alloc(&h->qinv, (size_t)h->m * h->m));
  RET(h->alloc(&h->qinv_df, (size_t)h->m * h->m));
  RET(h->alloc(&h->dy_prev, (size_t)h->lda + 64));
  RET(h->alloc(&h->ws_u, (size_t)h->lda + 64));
  RET(h->alloc(&h->ws_v, (size_t)h->lda + 64));
  RET(h->alloc(&h->ws_w, 2 * ((size_t)h->lda + 64)));
  RET(h->alloc(&h->ws_dots, 16));
  RET(h->alloc(&h->ws_X, (size_t)3 * h->m + 64));
  RET(h->alloc(&h->ws_Y, (size_t)h->m + 64));
  if (h->opt.sigma_rule == 1) {
    for (double** q : {&h->dy_aff, &h->dy_c, &h->p_aff, &h->p_c}) RET(h->alloc(q, (size_t)h->lda + 64));
    for (double** q : {&h->v_aff, &h->v_c}) RET(h->alloc(q, (size_t)h->npad));
  }
  RET(h->alloc(&h->gram_scratch, gram_df_scratch_floats(h->m, h->w, h->num_sms)));
  RET(h->alloc(&h->sweep_scratch, sweep_scratch_floats(h->m)));
  RET(h->alloc(&h->uw, (size_t)h->w));
  RET(h->alloc(&h->adwt_part, (size_t)h->adwt_parts * h->w));
  RET(h->alloc(&h->dinfo, 4));
  const int max_grid = std::max(h->plan.grid, h->use_rows ? std::max(h->rplan.grid, h->rplan_df.grid) : 0);
  h->alloc_grid = max_grid;
  RET(h->alloc(reinterpret_cast<char**>(&h->partials), (size_t)max_grid * 2 * h->lda * 8));
  RET(h->alloc(&h->gpart, (size_t)((max_grid + kGroup - 1) / kGroup) * 2 * h->lda));
  RET(h->alloc(&h->gtickets, kMaxGroups + 1));
  RET(h->alloc(&h->red_partials, (size_t)h->plan.grid * 2 + 2));
  RET(h->alloc(&h->tickets, 16));
  RET(h->alloc(&h->vpart, (size_t)h->num_sms * 8 + 64));
  RET(h->alloc(&h->sc, 1));
  CK(cudaMallocHost(&h->hsc, sizeof(DevScalars)));
  CK(cudaMallocHost(&h->hinfo, 4 * sizeof(int)));
  CK(cudaMallocHost(&h->hval, sizeof(double)));
  // cuSOLVER
  if (cusolverDnCreate(&h->sol) != CUSOLVER_STATUS_SUCCESS)
    return h->fail(LP_ERR_CUDA, "cusolverDnCreate failed");
  CS(cusolverDnSetStream(h->sol, h->st));
  CS(cusolverDnDgeqrf_bufferSize(h->sol, h->w, h->m, h->qr, h->w, &h->lwork_geqrf));
  CS(cusolverDnDpotrf_bufferSize(h->sol, CUBLAS_FILL_MODE_UPPER, h->m, h->rinv_cm, h->m, &h->lwork_potrf));
  if (cublasCreate(&h->blas) != CUBLAS_STATUS_SUCCESS) return h->fail(LP_ERR_CUDA, "cublasCreate failed");
  if (cublasSetStream(h->blas, h->st) != CUBLAS_STATUS_SUCCESS) return h->fail(LP_ERR_CUDA, "cublasSetStream failed");
  size_t dtr = 0, htr = 0;
  CS(cusolverDnXtrtri_bufferSize(h->sol, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, h->m,
                                 CUDA_R_64F, h->rinv_cm, h->m, &dtr, &htr));
  h->dwork_bytes = std::max<size_t>(std::max<size_t>((size_t)h->lwork_geqrf, (size_t)h->lwork_potrf) * sizeof(double), dtr) + 256;
  RET(h->alloc(reinterpret_cast<char**>(&h->dwork), h->dwork_bytes));
  h->hwork_bytes = std::max<size_t>(htr, 8);
  h->hwork = malloc(h->hwork_bytes);
  if (!h->hwork) return h->fail(LP_ERR_OOM, "host workspace");
  // norms of b and c for the stopping test
  CK(launch_dot(h->m, h->b, h->b, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[0], h->num_sms, h->st));
  CK(launch_dot(h->n, h->c, h->c, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[1], h->num_sms, h->st));
  RET(sync_read(h));
  h->bnorm = sqrt(h->hsc->pad[0]);
  h->cnorm = sqrt(h->hsc->pad[1]);
  if (!std::isfinite(h->bnorm) || !std::isfinite(h->cnorm))
    return h->fail(LP_ERR_ARG, "b or c contains NaN/Inf");
  if (h->opt.autotune && !h->sparse && h->dtype != LP_F64) RET(autotune_product(h));
  return LP_OK;
}

int lp_create(lp_handle** out, const lp_matrix* A, const double* b, const double* c,
              int32_t bc_on_device, const lp_options* opt) {
  if (!out) return LP_ERR_ARG;
  *out = nullptr;
  lp_handle* h = new (std::nothrow) lp_handle();
  if (!h) {
    g_create_error = "host allocation failed";
    return LP_ERR_OOM;
  }
  const int rc = guarded(&h->err, [&] { return create_impl(h, A, b, c, bc_on_device, opt); });
  if (rc != LP_OK) {
    g_create_error = h->err;
    lp_destroy(h);
    return rc;
  }
  g_create_error.clear();
  *out = h;
  return LP_OK;
}

// ---------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------
int lp_adat(lp_handle* h, const double* d2, const double* v, double* u, int32_t precision) {
  if (!h || !d2 || !v || !u) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  CK(cudaMemcpyAsync(h->d2d, d2, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
  h->d2df_valid = false;
  CK(launch_to_f32(h->n, h->d2d, h->d2f, 0, h->num_sms, h->st));
  CK(cudaMemcpyAsync(h->mb0, v, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemsetAsync(&h->sc->inner_done, 0, 2 * sizeof(int), h->st));
  RET(launch_adat(h, h->mb0, E_PLAIN, precision != 0, 0, h->mb1));
  CK(cudaMemcpyAsync(u, h->mb1, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, h->st));
  RET(sync_read(h));
  if (h->opt.profile) ev_flush(h);
  return LP_OK;
}

int lp_csr_to_csc(int32_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                  const void* val, int32_t dtype, int64_t* col_ptr, int32_t* row_idx, void* val_out) {
  if (m < 1 || n < 1 || n > INT32_MAX || nnz < 0 || !row_ptr || (nnz > 0 && (!col_idx || !val)) ||
      !col_ptr || (nnz > 0 && (!row_idx || !val_out)))
    return LP_ERR_ARG;
  if (dtype != LP_F64 && dtype != LP_F32 && dtype != LP_BF16) return LP_ERR_ARG;
  const int esz = dtype == LP_F64 ? 8 : (dtype == LP_F32 ? 4 : 2);
  std::string err;
  return guarded(&err, [&] {
    CscCopy conv;
    if (!csr_to_csc(m, n, nnz, row_ptr, col_idx, val, esz, &conv).empty()) return LP_ERR_ARG;
    std::memcpy(col_ptr, conv.ptr.data(), sizeof(int64_t) * ((size_t)n + 1));
    if (nnz > 0) {
      std::memcpy(row_idx, conv.idx.data(), sizeof(int32_t) * (size_t)nnz);
      std::memcpy(val_out, conv.val.data(), (size_t)esz * nnz);
    }
    return LP_OK;
  });
}

int lp_wait_probe(lp_handle* h, int64_t spin_cycles, int32_t complete) {
  if (!h || spin_cycles < 1 || spin_cycles > (1LL << 31) || (complete != 0 && complete != 1))
    return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  CK(launch_wait_probe(&h->sc->err, (long long)spin_cycles, complete, h->st));
  return sync_read(h);
}

int lp_residual_rhs(lp_handle* h, const double* x, const double* y, const double* s, int32_t mode,
                    double* r_p, double* r_d, double* p, double* out5) {
  if (!h || !x || !y || !s) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  h->state_valid = false;  // the handle's iterate is overwritten
  RET(copy_in(h, h->x, x, h->n, 1));
  RET(copy_in(h, h->s, s, h->n, 1));
  RET(copy_in(h, h->y, y, h->m, 1));
  RET(compute_mu(h));
  RET(residual_pass(h, mode == LP_FEASIBLE));
  if (r_p) RET(copy_out(h, r_p, h->rp, h->m, 1));
  if (r_d) RET(copy_out(h, r_d, h->rd, h->n, 1));
  if (p) RET(copy_out(h, p, h->p, h->m, 1));
  RET(sync_read(h));
  if (out5) {
    out5[0] = h->hsc->mu;
    out5[1] = h->hsc->cx;
    out5[2] = h->hsc->by;
    out5[3] = sqrt(h->hsc->rp2);
    out5[4] = sqrt(h->hsc->rd2);
  }
  return LP_OK;
}

int lp_sketch(lp_handle* h, const double* D, uint64_t seed, int64_t k, int32_t retry, double* adw,
              int64_t* w_out) {
  if (!h || !D || !adw || retry < 0 || retry >= kMaxRetry || k < 0) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  RET(copy_in(h, h->nb0, D, h->n, 1));
  CK(launch_sketch(h, h->nb0, 0, seed, k, retry));
  CK(cudaMemcpyAsync(adw, h->adw, sizeof(double) * (size_t)h->m * h->w, cudaMemcpyDeviceToDevice, h->st));
  RET(sync_read(h));
  if (w_out) *w_out = h->w;
  return LP_OK;
}

int lp_precond_apply(lp_handle* h, const double* adw, const double* r, double* z) {
  if (!h || !adw || !r || !z) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  CK(cudaMemcpyAsync(h->adw, adw, sizeof(double) * (size_t)h->m * h->w, cudaMemcpyDeviceToDevice, h->st));
  RET(factor(h));
  RET(copy_in(h, h->mb0, r, h->m, 1));
  RET(precond_gemvs(h, h->mb0, h->mb1, GH_NONE, 0));
  RET(copy_out(h, z, h->mb1, h->m, 1));
  RET(sync_read(h));
  return LP_OK;
}

int lp_directions(lp_handle* h, const double* x, const double* s, const double* rd, const double* dy,
                  const double* v, double mu, int32_t mode, double* dx, double* ds) {
  if (!h || !x || !s || !dy || !v || !dx || !ds) return LP_ERR_ARG;
  const bool feasible = mode == LP_FEASIBLE;
  if (!feasible && !rd) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  RET(copy_in(h, h->x, x, h->n, 1));
  RET(copy_in(h, h->s, s, h->n, 1));
  RET(copy_in(h, h->v, v, h->n, 1));
  if (!feasible) RET(copy_in(h, h->rd, rd, h->n, 1));
  RET(copy_in(h, h->dy, dy, h->m, 1));
  RET(set_scalar(h, &h->sc->mu, mu));
  RET(direction_pass(h, feasible));
  RET(copy_out(h, dx, h->dx, h->n, 1));
  RET(copy_out(h, ds, h->ds, h->n, 1));
  RET(sync_read(h));
  return LP_OK;
}

int lp_step_lengths(lp_handle* h, const double* x, const double* s, const double* dx, const double* ds,
                    int32_t mode, double res_ratio, double mu0, double* out2) {
  if (!h || !x || !s || !dx || !ds || !out2) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  RET(copy_in(h, h->x, x, h->n, 1));
  RET(copy_in(h, h->s, s, h->n, 1));
  RET(copy_in(h, h->dx, dx, h->n, 1));
  RET(copy_in(h, h->ds, ds, h->n, 1));
  const double inv_n = 1.0 / (double)h->n;
  CK(launch_dot(h->n, h->x, h->s, inv_n, h->vpart, h->tickets + 3, &h->sc->mu, h->num_sms, h->st));
  CK(launch_dot(h->n, h->x, h->ds, inv_n, h->vpart, h->tickets + 3, &h->sc->pad[0], h->num_sms, h->st));
  CK(launch_dot(h->n, h->s, h->dx, inv_n, h->vpart, h->tickets + 3, &h->sc->pad[1], h->num_sms, h->st));
  CK(launch_dot(h->n, h->dx, h->ds, inv_n, h->vpart, h->tickets + 3, &h->sc->c2, h->num_sms, h->st));
  RET(sync_read(h));
  RET(set_scalar(h, &h->sc->c1, h->hsc->pad[0] + h->hsc->pad[1]));
  CK(launch_step(h->n, h->x, h->s, h->dx, h->ds, h->opt.gamma, mode == LP_FEASIBLE, res_ratio, mu0,
                 h->vpart, h->tickets + 4, h->sc, h->num_sms, h->st));
  RET(sync_read(h));
  out2[0] = h->hsc->alpha_max;
  out2[1] = h->hsc->alpha_bar;
  return LP_OK;
}

int lp_get_history(lp_handle* h, lp_iter_record* recs, int32_t max_records) {
  if (!h || max_records < 0 || (max_records > 0 && !recs)) return LP_ERR_ARG;
  const int cnt = (int)h->history.size();
  for (int i = 0; i < std::min(cnt, (int)max_records); ++i) recs[i] = h->history[i];
  return cnt;
}

static int get_state_impl(lp_handle* h, lp_state* st, double* x, double* y, double* s, double* dy_prev,
                          int32_t io_on_device) {
  if (!h || !st || !x || !y || !s) return LP_ERR_ARG;
  h->err.clear();
  if (!h->state_valid) return h->fail(LP_ERR_ARG, "no solve state: no solve ended since the iterate was last set");
  RET(copy_out(h, x, h->x, h->n, io_on_device));
  RET(copy_out(h, y, h->y, h->m, io_on_device));
  RET(copy_out(h, s, h->s, h->n, io_on_device));
  if (dy_prev) RET(copy_out(h, dy_prev, h->dy_prev, h->m, io_on_device));
  CK(cudaStreamSynchronize(h->st));
  *st = h->last_state;
  if (!dy_prev) st->has_dy_prev = 0;
  return LP_OK;
}

static int set_state_impl(lp_handle* h, const lp_state* st, const double* x, const double* y, const double* s,
                          const double* dy_prev, int32_t io_on_device) {
  if (!h || !st || !x || !y || !s) return LP_ERR_ARG;
  h->err.clear();
  if (st->k < 0 || (st->mode != LP_FEASIBLE && st->mode != LP_INFEASIBLE) || st->reserved != 0 ||
      !(st->mu0 > 0) || !std::isfinite(st->mu0) || !(st->mu > 0) || !std::isfinite(st->mu) ||
      !(st->r0 >= 0) || !std::isfinite(st->r0) ||
      !(st->ratio_ref >= 0) || !std::isfinite(st->ratio_ref) || (st->has_dy_prev != 0 && st->has_dy_prev != 1) ||
      (st->has_dy_prev && !dy_prev))
    return h->fail(LP_ERR_ARG, "invalid state");
  h->state_valid = false;
  h->resume_pending = false;
  RET(copy_in(h, h->x, x, h->n, io_on_device));
  RET(copy_in(h, h->y, y, h->m, io_on_device));
  RET(copy_in(h, h->s, s, h->n, io_on_device));
  if (st->has_dy_prev) RET(copy_in(h, h->dy_prev, dy_prev, h->m, io_on_device));
  CK(cudaStreamSynchronize(h->st));
  h->resume = *st;
  h->opt.seed = st->seed;
  h->resume_pending = true;
  return LP_OK;
}

int lp_get_state(lp_handle* h, lp_state* st, double* x, double* y, double* s, double* dy_prev,
                 int32_t io_on_device) {
  return guarded(h ? &h->err : nullptr,
                 [&] { return get_state_impl(h, st, x, y, s, dy_prev, io_on_device); });
}

int lp_set_state(lp_handle* h, const lp_state* st, const double* x, const double* y, const double* s,
                 const double* dy_prev, int32_t io_on_device) {
  return guarded(h ? &h->err : nullptr,
                 [&] { return set_state_impl(h, st, x, y, s, dy_prev, io_on_device); });
}

static int check_guards_impl(lp_handle* h, int64_t* checked, int64_t* damaged) {
  if (!h || !checked || !damaged) return LP_ERR_ARG;
  h->err.clear();
  CK(cudaStreamSynchronize(h->st));
  std::vector<unsigned char> buf(lp_handle::kGuard);
  int64_t nchk = 0, nbad = 0;
  for (size_t i = 0; i < h->guarded_bufs.size(); ++i) {
    const lp_handle::GuardedBuf& g = h->guarded_bufs[i];
    for (int side = 0; side < 2; ++side) {
      const char* src = side ? g.base + lp_handle::kGuard + g.bytes : g.base;
      CK(cudaMemcpy(buf.data(), src, lp_handle::kGuard, cudaMemcpyDeviceToHost));
      ++nchk;
      bool ok = true;
      for (unsigned char c : buf) ok = ok && c == lp_handle::kGuardByte;
      if (!ok && nbad++ == 0)
        h->fail(LP_OK, "guard %s buffer %zu (%zu bytes) was overwritten", side ? "after" : "before", i, g.bytes);
    }
  }
  *checked = nchk;
  *damaged = nbad;
  return LP_OK;
}

int lp_release_cached_memory(void) {
  pool_release();
  return LP_OK;
}

int lp_check_guards(lp_handle* h, int64_t* checked, int64_t* damaged) {
  return guarded(h ? &h->err : nullptr, [&] { return check_guards_impl(h, checked, damaged); });
}

int lp_get_kernel_stats(lp_handle* h, lp_kernel_stats* st) {
  if (!h || !st) return LP_ERR_ARG;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return LP_ERR_CUDA;
  ev_flush(h);
  st->launches = h->k1_launches;
  st->ms = h->k1_ms;
  st->bytes_per_launch = h->sparse ? (int64_t)h->nnz * (h->esz + 4) + 8 * (h->n + 1) + 4 * h->n + 16 * (int64_t)h->m
                                    : (int64_t)h->m * h->n * h->esz + 4 * h->n + 2 * 8 * (int64_t)h->m;
  st->all_launches = g_launches.load() - h->launch_base;
  st->graph_replays = h->graph_replays;
  return LP_OK;
}

int lp_reset_kernel_stats(lp_handle* h) {
  if (!h) return LP_ERR_ARG;
  cudaStreamSynchronize(h->st);
  h->graph_replays = 0;
  ev_flush(h);
  h->k1_launches = 0;
  h->k1_ms = 0.0;
  h->launch_base = g_launches.load();
  return LP_OK;
}

// ---------------------------------------------------------------------------
// normal-equation solve (Algorithm 1 + eq. compv)
// ---------------------------------------------------------------------------
static int normal_solve_impl(lp_handle* h, const double* D, const double* p, const double* xs, int64_t k,
                    double tol_f, int32_t io_on_device, double* dy, double* v, lp_nsolve_info* info) {
  if (!h || !D || !p || !dy || k < 0) return LP_ERR_ARG;
  h->err.clear();
  RET(clear_status(h));
  RET(copy_in(h, h->nb0, D, h->n, io_on_device));
  RET(copy_in(h, h->p, p, h->m, io_on_device));
  CK(launch_square(h->n, h->nb0, h->d2d, h->num_sms, h->st));
  h->d2df_valid = false;
  CK(launch_to_f32(h->n, h->nb0, h->d2f, 1, h->num_sms, h->st));
  int retry = 0;
  h->ratio_ref = 0.0;  // a single solve: no earlier factor to compare with
  RET(sketch_and_factor(h, h->nb0, 0, k, &retry));
  int iters = 0;
  const SketchRef skr{h->nb0, 0, (long long)k, &retry};
  const int status = inner_solve_robust(h, tol_f, &iters, false, &skr);
  if (status < 0) return status;
  const double f_true = h->hsc->f_true, f0 = sqrt(std::max(h->hsc->rho0, 0.0));
  double vnorm = 0.0;
  if (xs && v) {
    RET(copy_in(h, h->nb1, xs, h->n, io_on_device));
    RET(correction(h, h->nb1, nullptr, k, retry));  // nb1 holds x o s
    CK(launch_dot(h->n, h->v, h->v, 1.0, h->vpart, h->tickets + 3, &h->sc->pad[2], h->num_sms, h->st));
    RET(copy_out(h, v, h->v, h->n, io_on_device));
  }
  RET(copy_out(h, dy, h->dy, h->m, io_on_device));
  RET(sync_read(h));
  if (xs && v) vnorm = sqrt(h->hsc->pad[2]);
  if (info) {
    info->inner_iterations = iters;
    info->retries = retry;
    info->f_norm = f_true;
    info->f0_norm = f0;
    info->v_norm = vnorm;
    info->lam_min = h->hsc->lam_min;
    info->lam_max = h->hsc->lam_max;
  }
  return status;
}

// ---------------------------------------------------------------------------
// the IPM (Algorithm 2 / Algorithm 3)
// ---------------------------------------------------------------------------
// NVTX ranges naming the phases of an outer iteration (shown by Nsight tools;
// without a tool attached a push or pop is a no-op)
struct PhaseRange {
  bool open = false;
  void next(const char* name) {
    end();
    nvtxRangePushA(name);
    open = true;
  }
  void end() {
    if (open) nvtxRangePop();
    open = false;
  }
  ~PhaseRange() { end(); }
};

static int solve_impl(lp_handle* h, double tol, int32_t mode, const double* x0, const double* y0,
             const double* s0, int32_t io_on_device, double* x, double* y, double* s,
             lp_result* info) {
  if (!h || !(tol > 0)) return LP_ERR_ARG;
  if (mode != LP_FEASIBLE && mode != LP_INFEASIBLE) return LP_ERR_ARG;
  h->err.clear();
  PhaseRange solve_range, phase;
  solve_range.next("lp_solve");
  const auto t_start = std::chrono::steady_clock::now();
  const bool feasible = mode == LP_FEASIBLE;
  h->history.clear();
  const bool resume = h->resume_pending;
  h->resume_pending = false;
  h->state_valid = false;
  if (resume) {
    if (x0 || y0 || s0) return h->fail(LP_ERR_ARG, "a resumed solve starts from its state: x0, y0, s0 must be null");
    if (mode != h->resume.mode) return h->fail(LP_ERR_ARG, "the state is from a solve in the other mode");
    if (h->resume.k > h->opt.k_max) return h->fail(LP_ERR_ARG, "the state's k exceeds k_max");
  }
  h->ratio_ref = resume ? h->resume.ratio_ref : 0.0;
  h->ws_have_prev = resume && h->resume.has_dy_prev != 0;
  lp_result res;
  std::memset(&res, 0, sizeof res);
  const long long n = h->n;
  const int m = h->m;
  // start point (a resumed solve finds its iterate in x, y, s already)
  if (!resume) {
    if (x0) RET(copy_in(h, h->x, x0, n, io_on_device));
    else CK(launch_fill(n, h->x, 1.0, h->num_sms, h->st));
    if (s0) RET(copy_in(h, h->s, s0, n, io_on_device));
    else CK(launch_fill(n, h->s, 1.0, h->num_sms, h->st));
    if (y0) RET(copy_in(h, h->y, y0, m, io_on_device));
    else CK(cudaMemsetAsync(h->y, 0, sizeof(double) * m, h->st));
  }
  if (feasible && !resume && (!x0 || !y0 || !s0))
    return h->fail(LP_ERR_NOT_FEASIBLE, "feasible mode needs x0, y0, s0");
  CK(cudaMemsetAsync(&h->sc->err, 0, sizeof(int), h->st));
  RET(compute_mu(h));
  CK(launch_min_prod(n, h->x, h->s, h->vpart, h->tickets + 5, &h->sc->pad[3], h->num_sms, h->st));
  RET(sync_read(h));
  const double mu_start = h->hsc->mu;
  if (!(mu_start > 0) || !(h->hsc->pad[3] > 0)) return h->fail(LP_ERR_ARG, "start needs x0 > 0 and s0 > 0");
  if (feasible && h->hsc->pad[3] < (1.0 - h->opt.gamma) * mu_start * (1.0 - 1e-9))
    return h->fail(LP_ERR_NOT_FEASIBLE, "start is not in N(gamma)");
  // mu_0 and ||r^0|| belong to the start of the whole solve, also when resumed
  const double mu0 = resume ? h->resume.mu0 : mu_start;
  double r0 = resume ? h->resume.r0 : 0.0;
  const int k_start = resume ? h->resume.k : 0;
  // a resumed solve continues with mu as the interrupted one had it (the
  // update's reduction), not x^T s / n summed afresh
  if (resume) CK(cudaMemcpyAsync(&h->sc->mu, &h->resume.mu, sizeof(double), cudaMemcpyHostToDevice, h->st));
  int status = LP_STATUS_MAX_ITER;
  double ms_res = 0, ms_sk = 0, ms_fac = 0, ms_in = 0, ms_cor = 0, ms_step = 0;
  auto now = [] { return std::chrono::steady_clock::now(); };
  auto ms_since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
  };
  bool pending = false;  // the last iteration's correction and step events are still to be read
  auto read_pending = [&]() -> int {
    if (!pending) return LP_OK;
    float a = 0.0f, b = 0.0f;
    CK(cudaEventElapsedTime(&a, h->ev_cor, h->ev_step));
    CK(cudaEventElapsedTime(&b, h->ev_step, h->ev_end));
    ms_cor += a;
    ms_step += b;
    pending = false;
    return LP_OK;
  };
  for (int k = k_start; k <= h->opt.k_max; ++k) {
    phase.next("residuals");
    // ---- step 3: residuals, mu, right-hand side, d^2 ----
    CK(cudaEventRecord(h->ev_res, h->st));  // after the previous step's kernels in stream order
    RET(residual_pass(h, feasible, h->opt.sigma_rule == 1 ? 0.0 : -1.0));
    CK(cudaEventRecord(h->ev_res_end, h->st));
    RET(sync_read(h));
    RET(read_pending());
    {
      float r = 0.0f;
      CK(cudaEventElapsedTime(&r, h->ev_res, h->ev_res_end));
      ms_res += r;
    }
    auto t0 = now();
    const DevScalars& S = *h->hsc;
    const double rp = sqrt(S.rp2), rd = sqrt(S.rd2);
    const StopMeasures sm = stop_measures(S.cx, S.by, S.rp2, S.rd2, h->bnorm, h->cnorm);
    const double gap = sm.gap, rp_rel = sm.rp_rel, rd_rel = sm.rd_rel;
    if (k > k_start && !h->history.empty()) {
      h->history.back().alpha_max = S.alpha_max;
      h->history.back().alpha_bar = S.alpha_bar;
    }
    lp_iter_record rec;
    std::memset(&rec, 0, sizeof rec);
    rec.k = k;
    rec.mu = S.mu;
    rec.rel_gap = gap;
    rec.rp_rel = rp_rel;
    rec.rd_rel = rd_rel;
    h->history.push_back(rec);
    if (k == 0) {
      r0 = sqrt(S.rp2 + S.rd2);
      if (feasible && (rp_rel > 1e-8 || rd_rel > 1e-8))
        return h->fail(LP_ERR_NOT_FEASIBLE, "start is not feasible (rel residuals %.2e, %.2e)", rp_rel, rd_rel);
    } else if (k > k_start && S.alpha_bar <= 0.0) {
      status = LP_STATUS_STALLED;
      res.outer_iterations = k;
      break;
    }
    res.outer_iterations = k;
    res.primal_obj = S.cx;
    res.dual_obj = S.by;
    res.rel_gap = gap;
    res.rp_rel = rp_rel;
    res.rd_rel = rd_rel;
    res.mu = S.mu;
    if (!std::isfinite(gap) || !std::isfinite(rp) || !std::isfinite(rd))
      return h->fail(LP_ERR_NUMERICAL, "non-finite residuals at iteration %d", k);
    if (stop_reached(sm, tol)) {
      status = LP_OK;
      break;
    }
    // mu has fallen far below what the gap test needs while a residual test
    // still fails: the residuals have stopped following (1 - alpha) r (the
    // inexact solves' floor); further iterations only drive mu to underflow
    if (S.mu <= 1e-3 * tol * mu0 && gap <= tol) {
      status = LP_STATUS_STALLED;
      break;
    }
    if (k == h->opt.k_max) break;
    const double mu = S.mu;
    const double res_ratio = feasible ? 0.0 : sqrt(S.rp2 + S.rd2) / r0;
    // ---- step 2 + Algorithm 1 steps 1-2: sketch and factor ----
    t0 = now();
    int retry = 0;
    phase.next("sketch_factor");
    RET(sketch_and_factor(h, h->d2d, 1, k, &retry));
    res.sketch_retries += retry;
    const int retry0 = retry;
    const SketchRef skr{h->d2d, 1, (long long)k, &retry};
    ms_fac += ms_since(t0);
    // ---- Algorithm 1 step 3: inner solve to the Lemma 4.4 level ----
    phase.next("inner_solve");
    t0 = now();
    const bool adaptive = h->opt.sigma_rule == 1;
    const double sig_lo = 0.1, sig_hi = 0.75;  // inside the analysis range (0, 4/5)
    const double tol_f = h->opt.inner_rule == LP_RULE_THEORY
                             ? theory_inner_tol(mu, n, h->opt.gamma, adaptive ? sig_lo : h->opt.sigma)
                             : 0.0;
    double sigma_k = h->opt.sigma;
    int iters = 0, ist = 0;
    const size_t mb = sizeof(double) * (size_t)m, nbytes = sizeof(double) * (size_t)n;
    if (!adaptive) {
      bool warm = false;
      RET(warm_start_prepare(h, mu / mu0, &warm));
      double tf = tol_f;
      if (warm && tf <= 0) tf = h->opt.tol_cg * sqrt(std::max(h->hsc->pad[1], 0.0));  // cold ||f^0||
      ist = inner_solve_robust(h, tf, &iters, warm, &skr);
      if (ist < 0) return ist;
      RET(warm_start_finish(h));
      ms_in += ms_since(t0);
      // ---- step 5: correction v, directions ----
      CK(cudaEventRecord(h->ev_cor, h->st));
      phase.next("correction");
      RET(correction(h, h->x, h->s, k, retry));
      RET(direction_pass(h, feasible));
    } else {
      // two right-hand sides on this sketch and Q: p(sigma) = p_aff + sigma p_c
      CK(cudaMemcpyAsync(h->p_aff, h->p, mb, cudaMemcpyDeviceToDevice, h->st));  // p(0)
      RET(residual_pass(h, feasible, 1.0));                                       // p(1)
      CK(launch_axpby(m, 1.0, h->p, -1.0, h->p_aff, h->p_c, h->num_sms, h->st));
      int it2 = 0;
      CK(cudaMemcpyAsync(h->p, h->p_aff, mb, cudaMemcpyDeviceToDevice, h->st));
      ist = inner_solve_robust(h, tol_f, &iters, false, &skr);
      if (ist < 0) return ist;
      RET(correction(h, h->x, h->s, k, retry));
      CK(cudaMemcpyAsync(h->dy_aff, h->dy, mb, cudaMemcpyDeviceToDevice, h->st));
      CK(cudaMemcpyAsync(h->v_aff, h->v, nbytes, cudaMemcpyDeviceToDevice, h->st));
      CK(cudaMemcpyAsync(h->p, h->p_c, mb, cudaMemcpyDeviceToDevice, h->st));
      const int ist2 = inner_solve_robust(h, tol_f, &it2, false, &skr);
      if (ist2 < 0) return ist2;
      RET(correction(h, h->x, h->s, k, retry));
      CK(cudaMemcpyAsync(h->dy_c, h->dy, mb, cudaMemcpyDeviceToDevice, h->st));
      CK(cudaMemcpyAsync(h->v_c, h->v, nbytes, cudaMemcpyDeviceToDevice, h->st));
      iters += it2;
      ist = std::max(ist, ist2);
      ms_in += ms_since(t0);
      CK(cudaEventRecord(h->ev_cor, h->st));
      phase.next("directions");
      // affine direction (sigma = 0) and its largest positivity-keeping step
      CK(cudaMemcpyAsync(h->dy, h->dy_aff, mb, cudaMemcpyDeviceToDevice, h->st));
      CK(cudaMemcpyAsync(h->v, h->v_aff, nbytes, cudaMemcpyDeviceToDevice, h->st));
      RET(direction_pass(h, feasible, 0.0));
      CK(launch_pos_step(n, h->x, h->s, h->dx, h->ds, h->vpart, h->tickets + 8, h->sc, h->num_sms, h->st));
      RET(sync_read(h));
      const double aa = h->hsc->alpha_aff;
      const double mu_aff = mu + h->hsc->c1 * aa + h->hsc->c2 * aa * aa;
      sigma_k = std::min(sig_hi, std::max(sig_lo, std::pow(std::max(mu_aff, 0.0) / mu, 3.0)));
      // the direction for sigma_k: dy, v (and dx, ds) are affine in sigma
      CK(launch_axpby(m, 1.0, h->dy_aff, sigma_k, h->dy_c, h->dy, h->num_sms, h->st));
      CK(launch_axpby(n, 1.0, h->v_aff, sigma_k, h->v_c, h->v, h->num_sms, h->st));
      RET(direction_pass(h, feasible, sigma_k));
    }
    {
      lp_iter_record& hr = h->history.back();
      hr.inner_iterations = iters;
      hr.retries = retry;
      hr.inner_status = ist;
      hr.factor_kind = h->factor_kind;
      hr.r_ratio = h->hsc->diag_min > 0 ? h->hsc->diag_max / h->hsc->diag_min : INFINITY;
      res.sketch_retries += retry - retry0;  // draws replaced by the inner solve's check
      hr.f_norm = h->hsc->f_true;
      hr.f0_norm = sqrt(std::max(h->hsc->rho0, 0.0));
      hr.tol_f = tol_f > 0 ? tol_f : h->opt.tol_cg * hr.f0_norm;
      hr.sigma = sigma_k;
    }
    res.inner_total += iters;
    res.inner_max = std::max(res.inner_max, iters);
    // ---- steps 6-8: step lengths and update ----
    phase.next("step");
    CK(cudaEventRecord(h->ev_step, h->st));
    CK(launch_step(n, h->x, h->s, h->dx, h->ds, h->opt.gamma, feasible ? 1 : 0, res_ratio, mu0,
                   h->vpart, h->tickets + 4, h->sc, h->num_sms, h->st));
    CK(launch_update(n, m, h->x, h->s, h->y, h->dx, h->ds, h->dy, h->sc, h->vpart, h->tickets + 6,
                     h->num_sms, h->st));
    CK(cudaEventRecord(h->ev_end, h->st));
    pending = true;
  }
  phase.end();
  CK(cudaStreamSynchronize(h->st));
  RET(read_pending());
  if (x) RET(copy_out(h, x, h->x, n, io_on_device));
  if (y) RET(copy_out(h, y, h->y, m, io_on_device));
  if (s) RET(copy_out(h, s, h->s, n, io_on_device));
  CK(cudaStreamSynchronize(h->st));
  h->last_state.k = res.outer_iterations;
  h->last_state.mode = mode;
  h->last_state.has_dy_prev = h->ws_have_prev ? 1 : 0;
  h->last_state.reserved = 0;
  h->last_state.mu0 = mu0;
  h->last_state.r0 = r0;
  h->last_state.ratio_ref = h->ratio_ref;
  h->last_state.seed = h->opt.seed;
  h->last_state.mu = res.mu;
  h->state_valid = true;
  res.status = status;
  res.ms_total = ms_since(t_start);
  res.ms_residual = ms_res;
  res.ms_sketch = ms_sk;
  res.ms_factor = ms_fac;
  res.ms_inner = ms_in;
  res.ms_correction = ms_cor;
  res.ms_step = ms_step;
  if (info) *info = res;
  return status;
}

static int set_warm_start_impl(lp_handle* h, int32_t mode, lp_mlp* model, float* rec_X, float* rec_T,
                      int32_t rec_capacity) {
  if (!h || mode < 0 || mode > 2 || (mode == 2 && !model) || rec_capacity < 0) return LP_ERR_ARG;
  if ((rec_X == nullptr) != (rec_T == nullptr)) return LP_ERR_ARG;
  if (model) {
    int in = 0, out = 0, hid = 0;
    mlp_dims(model, &in, &out, &hid);
    if (in != 3 * h->m || out != h->m) return LP_ERR_ARG;  // features 3m -> dy (m)
    const long long need = (long long)mlp_predict_scratch_floats(model);
    if (need > h->ws_hid_cap) {
      if (cudaStreamSynchronize(h->st) != cudaSuccess) return LP_ERR_CUDA;
      h->err.clear();
      if (h->alloc(&h->ws_hid, (size_t)need) != LP_OK) return LP_ERR_OOM;
      h->ws_hid_cap = need;
    }
  }
  h->ws_mode = mode;
  h->ws_model = model;
  h->ws_rec_X = rec_X;
  h->ws_rec_T = rec_T;
  h->ws_cap = rec_X ? rec_capacity : 0;
  h->ws_count = h->ws_props = h->ws_acc = 0;
  h->ws_have_prev = false;
  return LP_OK;
}

int lp_get_warm_start_stats(lp_handle* h, int64_t* recorded, int64_t* proposals, int64_t* accepted) {
  if (!h) return LP_ERR_ARG;
  if (recorded) *recorded = h->ws_count;
  if (proposals) *proposals = h->ws_props;
  if (accepted) *accepted = h->ws_acc;
  return LP_OK;
}

int lp_solve_batch(lp_handle* const* hs, int32_t count, double tol, int32_t mode,
                   int32_t io_on_device, double* const* x, double* const* y, double* const* s,
                   int32_t max_threads, lp_result* results) {
  if (!hs || count < 0 || !(tol > 0)) return LP_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return LP_ERR_ARG;
  for (int i = 0; i < count; ++i)
    for (int j = i + 1; j < count; ++j)
      if (hs[i] == hs[j]) return LP_ERR_ARG;  // one worker per handle
  std::vector<int> rc(count, LP_OK);
  std::vector<lp_result> res(count);
  std::atomic<int> next{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LP_ERR_CUDA;
  auto worker = [&]() {
    cudaSetDevice(dev);  // the current device is per host thread
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
      std::memset(&res[i], 0, sizeof(lp_result));
      rc[i] = lp_solve(hs[i], tol, mode, nullptr, nullptr, nullptr, io_on_device, x ? x[i] : nullptr,
                       y ? y[i] : nullptr, s ? s[i] : nullptr, &res[i]);
    }
  };
  int nt = max_threads > 0 ? max_threads : count;
  nt = std::max(1, std::min(std::min(nt, count), 64));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) {
    try {
      pool.emplace_back(worker);
    } catch (const std::system_error&) {
      break;  // fewer host threads: the ones running take the remaining LPs
    }
  }
  worker();
  for (auto& t : pool) t.join();
  if (results)
    for (int i = 0; i < count; ++i) results[i] = res[i];
  for (int i = 0; i < count; ++i)
    if (rc[i] < 0) return rc[i];
  return LP_OK;
}

// ---------------------------------------------------------------------------
// phase-1 primal start (Appendix "Feasible starting point")
// ---------------------------------------------------------------------------
namespace {
// element (row i, column j) of a host matrix of any storage dtype, sign-flipped
void put_neg(int dtype, void* dst, size_t idx, const void* src, size_t sidx, bool neg) {
  if (dtype == LP_F64) {
    const double v = static_cast<const double*>(src)[sidx];
    static_cast<double*>(dst)[idx] = neg ? -v : v;
  } else if (dtype == LP_F32) {
    const float v = static_cast<const float*>(src)[sidx];
    static_cast<float*>(dst)[idx] = neg ? -v : v;
  } else {
    const uint16_t v = static_cast<const uint16_t*>(src)[sidx];
    static_cast<uint16_t*>(dst)[idx] = neg ? (uint16_t)(v ^ 0x8000u) : v;  // bf16 sign bit
  }
}

void put_one(int dtype, void* dst, size_t idx) {
  if (dtype == LP_F64) static_cast<double*>(dst)[idx] = 1.0;
  else if (dtype == LP_F32) static_cast<float*>(dst)[idx] = 1.0f;
  else static_cast<uint16_t*>(dst)[idx] = 0x3F80u;  // bf16 1.0
}
}  // namespace

static int phase1_start_impl(const lp_matrix* A, const double* b, const lp_options* opt_in, double tol,
                             double* x0, lp_phase1_info* info) {
  if (!A || !b || !x0 || !(tol > 0) || A->on_device || A->m <= 0 || A->n <= 0) return LP_ERR_ARG;
  if (A->fmt != LP_DENSE_COLMAJOR && A->fmt != LP_CSC && A->fmt != LP_CSR) return LP_ERR_ARG;
  if (A->dtype != LP_F64 && A->dtype != LP_F32 && A->dtype != LP_BF16) return LP_ERR_ARG;
  if (!A->val) return LP_ERR_ARG;
  lp_matrix csc_view;
  CscCopy conv;
  if (A->fmt == LP_CSR) {  // rows sorted into columns on the host, as lp_create does
    if (!A->ptr || !A->idx || A->nnz < 0 || A->n > INT32_MAX) return LP_ERR_ARG;
    const int esz_in = A->dtype == LP_F64 ? 8 : (A->dtype == LP_F32 ? 4 : 2);
    if (!csr_to_csc(A->m, A->n, A->nnz, A->ptr, A->idx, A->val, esz_in, &conv).empty()) return LP_ERR_ARG;
    csc_view = *A;
    csc_view.fmt = LP_CSC;
    csc_view.ptr = conv.ptr.data();
    csc_view.idx = conv.idx.data();
    csc_view.val = conv.val.data();
    A = &csc_view;
  }
  if (A->fmt == LP_DENSE_COLMAJOR && A->ld < A->m) return LP_ERR_ARG;
  if (A->fmt == LP_CSC) {  // the structure is read on the host below: check it first
    if (!A->ptr || !A->idx || A->ptr[0] < 0) return LP_ERR_ARG;
    for (long long j = 0; j < A->n; ++j)
      if (A->ptr[j + 1] < A->ptr[j]) return LP_ERR_ARG;
  }
  const int m = A->m;
  const long long n = A->n, n1 = n + m;
  const int esz = A->dtype == LP_F64 ? 8 : (A->dtype == LP_F32 ? 4 : 2);
  lp_options opt;
  if (opt_in) opt = *opt_in;
  else lp_options_default(&opt);
  std::vector<char> neg(m);
  std::vector<double> b1(m), c1(n1, 0.0), zero_c(n, 0.0);
  double bnorm = 0.0;
  for (int i = 0; i < m; ++i) {
    neg[i] = b[i] < 0;
    b1[i] = std::fabs(b[i]);
    bnorm += b[i] * b[i];
  }
  bnorm = std::sqrt(bnorm);
  for (long long j = n; j < n1; ++j) c1[j] = 1.0;
  // [A | I] with the rows of negative b negated, same storage dtype and format
  lp_matrix A1 = *A;
  A1.n = n1;
  std::vector<char> val1;
  std::vector<int64_t> ptr1;
  std::vector<int32_t> idx1;
  if (A->fmt == LP_DENSE_COLMAJOR) {
    A1.ld = m;
    val1.assign((size_t)m * n1 * esz, 0);
    for (long long j = 0; j < n; ++j)
      for (int i = 0; i < m; ++i)
        put_neg(A->dtype, val1.data(), (size_t)j * m + i, A->val, (size_t)j * A->ld + i, neg[i] != 0);
    for (int i = 0; i < m; ++i) put_one(A->dtype, val1.data(), (size_t)(n + i) * m + i);
    A1.val = val1.data();
  } else {
    const int64_t nnz = A->ptr[n] - A->ptr[0];
    ptr1.resize(n1 + 1);
    idx1.resize(nnz + m);
    val1.assign((size_t)(nnz + m) * esz, 0);
    for (long long j = 0; j <= n; ++j) ptr1[j] = A->ptr[j] - A->ptr[0];
    for (int64_t e = 0; e < nnz; ++e) {
      const int32_t i = A->idx[A->ptr[0] + e];
      if (i < 0 || i >= m) return LP_ERR_ARG;
      idx1[e] = i;
      put_neg(A->dtype, val1.data(), (size_t)e, A->val, (size_t)(A->ptr[0] + e), neg[i] != 0);
    }
    for (int i = 0; i < m; ++i) {
      idx1[nnz + i] = i;
      put_one(A->dtype, val1.data(), (size_t)(nnz + i));
      ptr1[n + i + 1] = nnz + i + 1;
    }
    A1.val = val1.data();
    A1.ptr = ptr1.data();
    A1.idx = idx1.data();
    A1.nnz = nnz + m;
  }
  // phase-1 IPM from the usual infeasible start
  lp_handle* h1 = nullptr;
  int rc = lp_create(&h1, &A1, b1.data(), c1.data(), 0, &opt);
  if (rc != LP_OK) return rc;
  std::vector<double> x1(n1), y1(m), s1(n1);
  lp_result r1;
  rc = lp_solve(h1, tol, LP_INFEASIBLE, nullptr, nullptr, nullptr, 0, x1.data(), y1.data(), s1.data(), &r1);
  lp_destroy(h1);
  if (rc < 0) return rc;
  double z_sum = 0.0;
  for (int i = 0; i < m; ++i) z_sum += x1[n + i];
  lp_phase1_info inf{};
  inf.z_sum = z_sum;
  inf.outer_iterations = r1.outer_iterations;
  inf.inner_total = r1.inner_total;
  if (info) *info = inf;
  if (!(z_sum <= 1e-6 * (1.0 + bnorm))) return LP_ERR_NOT_FEASIBLE;
  // minimum-norm correction onto A x = b: x0 = x + A^T (A A^T)^{-1} (b - A x)
  lp_handle* h = nullptr;
  lp_options o0 = opt;
  o0.inner_rule = LP_RULE_RELATIVE;
  o0.tol_cg = 1e-13;
  rc = lp_create(&h, A, b, zero_c.data(), 0, &o0);
  if (rc != LP_OK) return rc;
  auto run = [&]() -> int {
    RET(copy_in(h, h->x, x1.data(), (size_t)n, 0));
    CK(launch_fill(n, h->s, 1.0, h->num_sms, h->st));
    CK(cudaMemsetAsync(h->y, 0, sizeof(double) * m, h->st));
    CK(cudaMemsetAsync(h->v, 0, sizeof(double) * h->npad, h->st));
    RET(set_scalar(h, &h->sc->mu, 0.0));
    RET(residual_pass(h, true));                                  // rp = A x - b
    CK(launch_axpby(m, -1.0, h->rp, 0.0, h->rp, h->p, h->num_sms, h->st));  // p = b - A x
    CK(launch_fill(n, h->d2d, 1.0, h->num_sms, h->st));               // D = I
    CK(launch_to_f32(n, h->d2d, h->d2f, 0, h->num_sms, h->st));
    h->d2df_valid = false;
    int retry = 0;
    RET(sketch_and_factor(h, h->d2d, 1, 0, &retry));
    int iters = 0;
    const SketchRef skr{h->d2d, 1, 0, &retry};
    const int st = inner_solve_robust(h, 0.0, &iters, false, &skr);  // dy = (A A^T)^{-1} p
    if (st < 0) return st;
    RET(direction_pass(h, true));                                   // ds = -A^T dy
    CK(launch_axpby(n, 1.0, h->x, -1.0, h->ds, h->x, h->num_sms, h->st));  // x0 = x - ds
    RET(residual_pass(h, true));                                    // ||A x0 - b||
    RET(copy_out(h, x0, h->x, (size_t)n, 0));
    RET(sync_read(h));
    inf.residual = std::sqrt(h->hsc->rp2);
    return LP_OK;
  };
  rc = run();
  lp_destroy(h);
  if (rc < 0) return rc;
  double xmin = INFINITY;
  for (long long j = 0; j < n; ++j) xmin = std::min(xmin, x0[j]);
  inf.x0_min = xmin;
  if (info) *info = inf;
  return xmin > 0.0 ? LP_OK : LP_ERR_NUMERICAL;
}

int lp_normal_solve(lp_handle* h, const double* D, const double* p, const double* xs, int64_t k,
                    double tol_f, int32_t io_on_device, double* dy, double* v, lp_nsolve_info* info) {
  return guarded(h ? &h->err : nullptr,
                 [&] { return normal_solve_impl(h, D, p, xs, k, tol_f, io_on_device, dy, v, info); });
}

int lp_solve(lp_handle* h, double tol, int32_t mode, const double* x0, const double* y0,
             const double* s0, int32_t io_on_device, double* x, double* y, double* s,
             lp_result* info) {
  return guarded(h ? &h->err : nullptr,
                 [&] { return solve_impl(h, tol, mode, x0, y0, s0, io_on_device, x, y, s, info); });
}

int lp_set_warm_start(lp_handle* h, int32_t mode, lp_mlp* model, float* rec_X, float* rec_T,
                      int32_t rec_capacity) {
  return guarded(h ? &h->err : nullptr,
                 [&] { return set_warm_start_impl(h, mode, model, rec_X, rec_T, rec_capacity); });
}

int lp_phase1_start(const lp_matrix* A, const double* b, const lp_options* opt_in, double tol,
                    double* x0, lp_phase1_info* info) {
  return guarded(nullptr, [&] { return phase1_start_impl(A, b, opt_in, tol, x0, info); });
}

}  // extern "C"
