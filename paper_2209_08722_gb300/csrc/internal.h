// Declarations shared by the translation units of the CUDA library.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <utility>

#include "common.cuh"
#include "stream.cuh"

struct lp_mlp;  // the warm-start model (mlp.cu; opaque in the C ABI)

namespace lpk {

// kernels launched by this library since load (cuSOLVER's own kernels excluded)
extern std::atomic<long long> g_launches;

struct StreamPlan {
  int nb = 0, ntiles = 0, stages = 0, grid = 0, smem = 0, smem8 = 0;
  bool ok = false;
};

StreamPlan make_stream_plan(int m, long long n, int lda, int esz, int num_sms, int tc_bytes);
StreamPlan make_stream_plan_ex(int m, long long n, int lda, int esz, int num_sms, int tc_bytes, int target,
                               int max_stages);
int fused_vpl(int lda, int esz);
cudaError_t launch_stream(int dtype, bool fp64_acc, int mode, const StreamArgs& a,
                          const StreamPlan& p, cudaStream_t st);
// pdl: launch with programmatic stream serialization (see pdl_wait in common.cuh)
cudaError_t launch_adat_fused(int dtype, const StreamArgs& a, const StreamPlan& p, cudaStream_t st,
                              bool pdl = false);

// kernel launch with programmatic stream serialization when pdl is set
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
// FP64 n-vectors <-> FP32 pairs for the double-float streaming passes
struct DfPackArgs {
  const double* src[4];
  float2* dst[4];
  int k;
  long long n;
};
struct DfUnpackArgs {
  int mode;  // 0: residual pass (r_d, d2, fl32(d2)); 1: direction pass (dx, ds)
  long long n;
  const float2* df0;
  const float2* df1;
  double* out0;
  double* out1;
  float* outf;
  const double* x;
  const double* s;
  const double* c;
  DevScalars* sc;
  double* part;     // [2 x grid] partial column sums
  unsigned* ticket;
};
cudaError_t launch_df_pack(const DfPackArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_df_unpack(const DfUnpackArgs& a, int num_sms, cudaStream_t st);

// the warm-start model's forward pass for one sample on stream st into
// scratch of mlp_predict_scratch_floats floats (mlp.cu)
int mlp_predict(::lp_mlp* M, const float* X, float* scratch, float* Y, cudaStream_t st);
size_t mlp_predict_scratch_floats(const ::lp_mlp* M);
void mlp_dims(const ::lp_mlp* M, int* in, int* out, int* hid);
// the model's contractions (mlp_gemm.cu): C = op(A) op(B), column-major FP32,
// split-TF32 on the tcgen05 tensor cores; y-partials of a column-major GEMV
// over gemv_slices(cols) column slices ([slice][rows])
cudaError_t launch_gemm_tf32x3(bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B,
                               int ldb, float* C, int ldc, int* err, cudaStream_t st);
int gemv_slices(int cols);
cudaError_t launch_gemv_cm(int rows, int cols, const float* W, const float* x, float* part, cudaStream_t st);

// raise (never lower) a kernel's dynamic shared-memory limit; thread-safe
cudaError_t ensure_smem(const void* func, int bytes);

// Row-split streaming kernels for tall columns (stream_rows.cu): FP32 M_ADAT
// (df = false) and the double-float passes M_ADAT, M_RESID, M_DIR (df = true)
// with their own tile width (nb = 4 x column groups) and stage count.
struct RowsPlan {
  int rpt = 0, nb = 0, ntiles = 0, stages = 0, grid = 0, smem = 0;
  bool ok = false;
};
RowsPlan make_rows_plan(int lda, long long n, int esz, int num_sms, bool df);
cudaError_t launch_rows(int dtype, bool df, int mode, const StreamArgs& a, const RowsPlan& p,
                        cudaStream_t st, bool pdl);

// double-float streaming passes (M_ADAT, M_RESID, M_DIR) for FP32/BF16 storage
cudaError_t launch_stream_df(int dtype, int mode, const StreamArgs& a, const StreamPlan& p,
                             cudaStream_t st);
bool stream_df_supported(int mode, int lda, int esz, const StreamPlan& p);

int sparse_grid(int num_sms);
// deterministic two-pass form (CSC column pass + CSR row-segment pass + one-CTA
// epilogue); a carries the CSR arrays, segments, column scalars and segment sums
constexpr int kSegNnz = 4096;  // CSR entries per row segment at most
int sparse2_col_grid(long long n, int num_sms);
cudaError_t launch_sparse2(int dtype, bool fp64, int mode, const StreamArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_sparse_sketch(int dtype, const long long* cp, const int* ri, const void* val,
                                 long long n, const double* dvec, int is_d2, uint64_t seed,
                                 long long k, int retry, int s_blocks, int w, double* adw, int m,
                                 int num_sms, cudaStream_t st);
cudaError_t launch_gauss_sketch(int dtype, const void* A, int lda, int m, long long n,
                                const double* dvec, int is_d2, uint64_t seed, long long k, int retry,
                                int w, double* adw, int tensor, int* err, int num_sms,
                                cudaStream_t st);
cudaError_t launch_gauss_tc(int dtype, const void* A, int lda, int m, long long n, const double* dvec,
                            int is_d2, uint64_t s_kr, int w, float inv_sqrt_w, double* adw, int* err,
                            int num_sms, cudaStream_t st);
cudaError_t launch_gauss_v(long long n, const double* x, const double* s, const double* dvec,
                           int is_d2, const double* u, uint64_t seed, long long k, int retry, int w,
                           double scale, double* v, int num_sms, cudaStream_t st);
// Gram (ADW)(ADW)^T in double-float: upper triangle of the column-major m x m
// g; scratch holds gram_df_scratch_floats() floats
void gram_df_split(int m, int w, int num_sms, int* ks, int* kper);
size_t gram_df_scratch_floats(int m, int w, int num_sms);
cudaError_t launch_gram_df(const double* x, int m, int w, float* scratch, double* g, int num_sms,
                           cudaStream_t st);

// Q^{-1} from the upper triangle of the column-major Gram g by the blocked
// symmetric sweep in double-float; rank check into sc (|R_ii| range)
size_t sweep_scratch_floats(int m);
// st_aux, ev_x, ev_p (nullable): second stream and events on which the pivot
// kernels overlap the tile kernels; without them everything runs on st
cudaError_t launch_sweep_inverse(const double* g, int m, float* scratch, double* qinv, float2* qinv_df,
                                 DevScalars* sc, double rank_tol, int num_sms, cudaStream_t st,
                                 cudaStream_t st_aux = nullptr, cudaEvent_t ev_x = nullptr,
                                 cudaEvent_t ev_p = nullptr);

// scratch of the dense CountSketch: bucket sizes/offsets/cursors (w + 1 each),
// bucket lists (n s), per-column scales (n)
struct CsWork {
  int* count = nullptr;
  int* base = nullptr;
  int* cursor = nullptr;
  int* list = nullptr;
  double* sc64 = nullptr;
  float2* scdf = nullptr;
};
constexpr int kCsMaxW = 40960;  // the bucket histogram lives in shared memory
cudaError_t launch_countsketch(int dtype, const void* A, int lda, int m, long long n,
                               const double* dvec, int is_d2, uint64_t seed, long long k,
                               int retry, int s_blocks, int w, double* adw, const CsWork& ws,
                               int* err, int num_sms, cudaStream_t st);
// CountSketch of a CSC A summed per bucket in a fixed order (bitwise
// reproducible); needs the CsWork lists, w <= kCsMaxW and m <= kSpMaxRows
constexpr int kSpMaxRows = 1 << 20;
cudaError_t launch_sparse_countsketch(int dtype, const long long* cp, const int* ri, const void* val,
                                      long long n, const double* dvec, int is_d2, uint64_t seed, long long k,
                                      int retry, int s_blocks, int w, double* adw, int m, const CsWork& ws,
                                      int num_sms, cudaStream_t st);
cudaError_t launch_v_gather(long long n, const double* x, const double* s, const double* u,
                            uint64_t seed, long long k, int retry, int s_blocks, int w, double scale,
                            double* v, int num_sms, cudaStream_t st);

enum GemvEpiHost : int {
  GH_NONE = 0, GH_PCG_INIT = 1, GH_PCG_B = 2, GH_REFRESH = 3, GH_CHEB_INIT = 4, GH_CHEB_B = 5,
  GH_CHEB_REFRESH = 6, GH_PCG_B_LAST = 7
};
cudaError_t launch_gemv_tri(const double* M, int m, int lower, const double* x, double* y, int epi,
                            int skip_level, double* r, double* p, double* dy, DevScalars* sc,
                            unsigned* ticket, int* err, int t_max, double* coef, int num_sms,
                            cudaStream_t st, const double* y_add = nullptr,
                            const float2* Mdf = nullptr, bool pdl = false);
cudaError_t launch_gemv_rows(const double* M, int rows, int cols, const double* x, const double* y0,
                             double alpha, double beta, double* y, int num_sms, cudaStream_t st);
cudaError_t launch_cheb_pre(int m, double* dy, const double* dir, DevScalars* sc, cudaStream_t st);
cudaError_t launch_adwt(const double* adw, int m, int w, const double* g, double* part, int max_parts,
                        double* out, int num_sms, cudaStream_t st);
cudaError_t launch_dot(long long n, const double* x, const double* y, double scale, double* part,
                       unsigned* ticket, double* out, int num_sms, cudaStream_t st);
cudaError_t launch_step(long long n, const double* x, const double* s, const double* dx,
                        const double* ds, double gamma, int feasible, double res_ratio, double mu0,
                        double* part, unsigned* ticket, DevScalars* sc, int num_sms, cudaStream_t st);
cudaError_t launch_update(long long n, int m, double* x, double* s, double* y, const double* dx,
                          const double* ds, const double* dy, DevScalars* sc, double* part,
                          unsigned* ticket, int num_sms, cudaStream_t st);
cudaError_t launch_fill(long long n, double* x, double v, int num_sms, cudaStream_t st);
// one thread waits (mbar_wait_for, limit in clock64 cycles) on a shared-memory
// mbarrier that it completes first when `complete` is set, and that nothing
// completes otherwise; a wait that gives up sets *err = ERR_TIMEOUT
cudaError_t launch_wait_probe(int* err, long long limit, int complete, cudaStream_t st);
cudaError_t launch_axpby(long long n, double alpha, const double* x, double beta, const double* y,
                         double* out, int num_sms, cudaStream_t st);
cudaError_t launch_ws_features(int m, const double* dy_prev, int have_prev, const double* u,
                               const DevScalars* sc, float* X, cudaStream_t st);
cudaError_t launch_ws_scale(int m, int dir, const float* yf, const double* in, const DevScalars* sc,
                            double* out, float* of, cudaStream_t st);
cudaError_t launch_pos_step(long long n, const double* x, const double* s, const double* dx,
                            const double* ds, double* part, unsigned* ticket, DevScalars* sc, int num_sms,
                            cudaStream_t st);
cudaError_t launch_min_prod(long long n, const double* x, const double* y, double* part,
                            unsigned* ticket, double* out, int num_sms, cudaStream_t st);
cudaError_t launch_to_f32(long long n, const double* x, float* y, int square, int num_sms,
                          cudaStream_t st);
cudaError_t launch_square(long long n, const double* x, double* y, int num_sms, cudaStream_t st);
cudaError_t launch_factor_utils(int which, const double* a, int w, int m, double* b, DevScalars* sc,
                                double rank_tol, int num_sms, cudaStream_t st);

}  // namespace lpk
