/*
 * lp_sketch_ipm.h -- C ABI of the GB300 sketched inexact interior-point LP solver.
 *
 * Problem (arXiv 2209.08722, Section 1, eq. primal / eq. dual):
 *     min c^T x  s.t.  A x = b, x >= 0        max b^T y  s.t.  A^T y + s = c, s >= 0
 * with A in R^{m x n}, m << n, full row rank (Section 1).
 *
 * Every outer iteration solves the normal equations A D^2 A^T dy = p (eq. normal,
 * D = X^{1/2} S^{-1/2}) inexactly: a sparse-embedding (CountSketch) sketch A D W
 * (Section 2, eq. pdprec), a factorisation of that sketch giving the
 * preconditioner Q = A D W W^T D A^T (eq. pdprecond, Algorithm 1 steps 1-2),
 * preconditioned CG or Chebyshev iteration run to the inexactness bound
 * (Algorithm 1 step 3, Lemma 4.4), and the correction vector v of eq. (compv).
 * The outer loop is Algorithm 2 (feasible start) or Algorithm 3 (infeasible start).
 *
 * Conventions for every entry point:
 *   - Return value: 0 = LP_OK; negative = error (LP_ERR_*); positive = a
 *     completed call with a warning status (LP_STATUS_*, LP_WARN_*).  After an
 *     error, lp_last_error(h) gives a one-line message.  No C++ exception
 *     crosses this interface: a failed host allocation returns LP_ERR_OOM.
 *   - Ownership: the handle owns all device memory it allocates.  Caller
 *     buffers are never retained: lp_create copies A, b, c; outputs are written
 *     into caller-allocated buffers.
 *   - Host or device pointers: calls that take an `on_device` flag accept host
 *     pointers (0) or device pointers on the handle's device (1).  Calls in the
 *     "kernel-level" section take DEVICE pointers only.
 *   - All vectors are FP64 unless stated.  A handle is not thread-safe; calls on
 *     one handle are ordered on its stream and every call returns after its
 *     work completed (the host synchronises the stream).
 */
#ifndef LP_SKETCH_IPM_H
#define LP_SKETCH_IPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque solver handle: owns the device copy of A, b, c and every workspace. */
typedef struct lp_handle lp_handle;

/* ---- status codes ------------------------------------------------------- */
#define LP_OK                   0
#define LP_ERR_ARG             -1  /* invalid argument (sizes, pointers, options) */
#define LP_ERR_CUDA            -2  /* a CUDA runtime / cuBLAS / cuSOLVER call failed */
#define LP_ERR_OOM             -3  /* device allocation failed */
#define LP_ERR_SKETCH_RANK     -4  /* A D W rank deficient after every redraw (Lemma 4.1) */
#define LP_ERR_NOT_FEASIBLE    -5  /* feasible mode: start not strictly feasible / not in N(gamma) */
#define LP_ERR_NUMERICAL       -6  /* NaN/Inf or a breakdown in a reduction */
#define LP_ERR_DEVICE_TIMEOUT  -7  /* a bounded device-side wait gave up */
#define LP_ERR_UNSUPPORTED     -8  /* valid request the library does not implement */
#define LP_STATUS_MAX_ITER      1  /* lp_solve: k_max outer iterations reached */
#define LP_WARN_INNER_MAXIT     2  /* an inner solve stopped at t_max */
#define LP_STATUS_STALLED       3  /* lp_solve: step length reached zero, or mu fell far below the gap
                                      tolerance while a residual test still fails */

/* ---- matrix description -------------------------------------------------- */
typedef enum { LP_DENSE_COLMAJOR = 0, LP_CSC = 1, LP_CSR = 2 } lp_format;
typedef enum { LP_F64 = 0, LP_F32 = 1, LP_BF16 = 2 } lp_dtype;

typedef struct {
    int32_t m;            /* rows (constraints) */
    int64_t n;            /* columns (variables) */
    int32_t fmt;          /* lp_format */
    int32_t dtype;        /* lp_dtype of the stored values; the LP solved is the one
                             with these (rounded) values */
    const void* val;      /* dense: column j at val + j*ld; CSC/CSR: nnz values */
    int64_t ld;           /* dense: leading dimension (>= m); ignored for CSC/CSR */
    const int64_t* ptr;   /* CSC: n+1 column pointers; CSR: m+1 row pointers (ptr[0] = 0) */
    const int32_t* idx;   /* CSC: nnz row indices in [0, m); CSR: nnz column indices in
                             [0, n) (so n < 2^31) */
    int64_t nnz;          /* CSC/CSR: number of stored entries */
    int32_t on_device;    /* 1: val/ptr/idx are device pointers */
} lp_matrix;

/* ---- options -------------------------------------------------------------- */
enum { LP_SKETCH_COUNT = 0, LP_SKETCH_GAUSS = 1 };
enum { LP_INNER_CG = 0, LP_INNER_CHEBYSHEV = 1 };
enum { LP_RULE_THEORY = 0, LP_RULE_RELATIVE = 1 };
enum { LP_FEASIBLE = 0, LP_INFEASIBLE = 1 };

typedef struct {
    double sigma;          /* centering parameter in (0, 1); the analysis of Algorithms 2-3
                              takes it in (0, 4/5); 0.5 */
    double gamma;          /* neighbourhood N(gamma) width, (0, 1) (eq. neigh); 0.999 */
    double tol_cg;         /* relative inner tolerance for LP_RULE_RELATIVE (Section 7); 1e-5 */
    int32_t inner_rule;    /* LP_RULE_THEORY: ||f|| <= gamma sigma sqrt(mu)/(4 sqrt(3n)) (Lemmas 4.2, 4.4) */
    int32_t sketch;        /* LP_SKETCH_COUNT (Section 2) or LP_SKETCH_GAUSS (Section 6) */
    int32_t s;             /* nonzeros per row of a CountSketch W (1..16); 2 */
    int32_t inner;         /* LP_INNER_CG or LP_INNER_CHEBYSHEV (Section 3) */
    int32_t refine_every;  /* FP64 true-residual refresh every k inner steps; 8 */
    int32_t k_max;         /* outer iteration limit; 200 */
    int32_t t_max;         /* inner iteration limit per outer iteration; 500 */
    int32_t v_correction;  /* 1: apply eq. (compv); 0: v = 0 (Table 2 ablation) */
    int32_t cheb_lanczos;  /* CG steps used to estimate the Chebyshev interval; 10 */
    int32_t profile;       /* 1: time the hot product kernel with CUDA events: one
                              block of 8 CG steps in 8 runs without the overlapped
                              (programmatic) launches, and its products but the
                              first are timed; 0 */
    double w_factor;       /* sketch width w = w_factor * m when w == 0, in (0, 1e6]; 4.0 */
    int64_t w;             /* explicit sketch width (rounded up to a multiple of s), or 0;
                              the width used must be >= m (Lemma 4.1 needs rank m) */
    uint64_t seed;         /* seed of the sketch generator; 0 */
    void* stream;          /* cudaStream_t to run on, or NULL for a private stream
                              (the factor also uses a private second stream, joined
                              back to this one by events before the factor ends) */
    int32_t tensor_sketch; /* Gaussian sketch with FP32/BF16 A: 1 = tcgen05 tensor-core GEMM,
                              0 = FP32 SIMT kernel; 1 */
    int32_t precondition;  /* 1 = the paper's method (sketch, Q^{-1}, correction v);
                              0 = the standard IPM of Section 7's comparison: unpreconditioned
                              CG on eq. normal (Q = I), no sketch, v = 0; 1 */
    int32_t sigma_rule;    /* 0 = fixed sigma (Algorithms 2-3); 1 = two right-hand sides per
                              outer iteration on one sketch and Q: p(sigma) = p(0) + sigma
                              (p(1) - p(0)) is affine in sigma, so are dy, v and the
                              directions; sigma = clip((mu_aff/mu)^3, 0.1, 0.75) from the
                              affine direction's largest positivity-keeping step; 0 */
    int32_t graphs;        /* 1: each block of refine_every inner steps (products, preconditioner
                              GEMVs, the true-residual refresh) is captured once per handle as
                              a CUDA graph and replayed with one launch; the kernels and their
                              results are the same as with plain launches (0); 1 */
    int32_t autotune;      /* 1: lp_create times the inner-loop product's candidate tile shapes
                              (warp-per-column kernel with 16/32/64 KB tiles and 2-4 stages,
                              the row-split kernel where the rows allow) on A and keeps the
                              fastest, cached per process by (dtype, leading dimension, n), so
                              later handles of that shape reuse it untimed; the choice changes
                              the product's summation order (results agree with autotune = 0 to
                              rounding); 0 */
    int32_t guard;         /* 1: every device workspace buffer of the handle is allocated with a
                              256-byte guard region before and after it, filled with the byte
                              0xA5; lp_check_guards reports regions that changed (a write past
                              a buffer's ends: the stand-in for a device memory checker).  The
                              results are the same as with guard = 0; 0 */
} lp_options;

/* ---- results -------------------------------------------------------------- */
typedef struct {
    int32_t status;             /* LP_OK (optimal to tol), LP_STATUS_*, or an error */
    int32_t outer_iterations;
    int64_t inner_total;        /* sum of inner iterations */
    int32_t inner_max;          /* max inner iterations of one outer iteration */
    int32_t sketch_retries;     /* total redraws of W: rank failures and failed Ritz checks */
    double primal_obj;          /* c^T x */
    double dual_obj;            /* b^T y */
    double rel_gap;             /* |c^T x - b^T y| / (1 + |c^T x|) */
    double rp_rel;              /* ||A x - b|| / (1 + ||b||) */
    double rd_rel;              /* ||A^T y + s - c|| / (1 + ||c||) */
    double mu;                  /* final x^T s / n */
    double ms_total;            /* wall time of the call */
    /* time per phase, summed over the outer iterations: residual, correction
     * (with the directions) and step are the device time between stream
     * events around their kernels; sketch + factor and the inner solve are
     * host wall time (they end with host decisions); ms_sketch is 0 (the
     * sketch is inside ms_factor) */
    double ms_residual, ms_sketch, ms_factor, ms_inner, ms_correction, ms_step;
} lp_result;

typedef struct {
    int32_t inner_iterations;   /* CG / Chebyshev iterations taken */
    int32_t retries;            /* sketch redraws (rank failures) */
    double f_norm;              /* ||f^(t)|| = sqrt(r^T Q^{-1} r), r = p - A D^2 A^T dy (FP64) */
    double f0_norm;             /* ||Q^{-1/2} p|| */
    double v_norm;              /* ||v|| (0 when v was not requested) */
    double lam_min, lam_max;    /* Chebyshev interval used (0 for CG) */
} lp_nsolve_info;

typedef struct {
    int64_t launches;           /* hot product kernel launches timed since the last reset */
    double ms;                  /* their summed CUDA-event duration */
    int64_t bytes_per_launch;   /* algorithmic bytes of one launch (A + d^2 + in/out vectors) */
    int64_t all_launches;       /* every kernel this library launched since the last reset
                                   (library-wide counter, the kernels of replayed graphs
                                   included; cuSOLVER's kernels not included) */
    int64_t graph_replays;      /* blocks of inner steps replayed from a CUDA graph (opt.graphs) */
} lp_kernel_stats;

/* One record per outer iteration of the last lp_solve (iteration log). */
typedef struct {
    int32_t k;                  /* outer iteration index */
    int32_t inner_iterations;   /* inner iterations of this outer iteration */
    int32_t retries;            /* sketch redraws */
    int32_t inner_status;       /* LP_OK or LP_WARN_INNER_MAXIT */
    double mu, rel_gap, rp_rel, rd_rel;   /* at the start of the iteration */
    double f_norm;              /* final ||f|| of the inner solve */
    double f0_norm;             /* ||Q^{-1/2} p|| */
    double tol_f;               /* the inner target used */
    double alpha_max, alpha_bar;
    double sigma;               /* centering parameter used */
    double r_ratio;             /* max |R_ii| / min |R_ii| of the factor in use (a lower
                                   bound on kappa(A D W)) */
    int32_t factor_kind;        /* factor in use at the end of the inner solve: 0 the
                                   double-float sweep of the Gram, 1 FP64 Cholesky of
                                   the Gram, 2 FP64 QR of (A D W)^T */
    int32_t reserved;           /* 0 */
} lp_iter_record;

/* ---- lifecycle -------------------------------------------------------------- */

/* Fills `opt` with the defaults listed above. */
void lp_options_default(lp_options* opt);

/* Copies A (dense column-major, CSC or CSR), b (m) and c (n) to the device in
 * the handle's layout and allocates every workspace the solver needs.  The
 * sparse kernels stream A by columns (the product A D^2 A^T v of eq. normal
 * gathers a_j^T v and scatters a_j t_j per column), so a CSR matrix is sorted
 * into CSC on the host (a device CSR is first read back); each column's entries
 * then come in increasing row order, and the handle is the same as the one
 * created from the equivalent CSC input with sorted rows.  CSR and CSC values
 * are FP32 or FP64.  `bc_on_device` says where b and c live.  Errors:
 * LP_ERR_ARG (sizes, m > n, bad CSC or CSR structure, bad options, a sketch
 * width below m), LP_ERR_OOM, LP_ERR_CUDA, LP_ERR_UNSUPPORTED (a shape the
 * library's kernels do not cover, BF16 sparse values, the Gaussian sketch with
 * a sparse A).  On error *h is NULL and lp_create_error() says why.  Errors in
 * the arguments themselves (pointers, sizes, the CSC or CSR structure of a host
 * matrix, the options, the sketch width) are reported before any CUDA call is
 * made; the structure of a device CSR is checked after it is read back;
 * NaN/Inf in b or c is found on the device. */
int lp_create(lp_handle** h, const lp_matrix* A, const double* b, const double* c,
              int32_t bc_on_device, const lp_options* opt);

/* The CSR -> CSC sort that lp_create applies to an LP_CSR matrix, offered on
 * its own (host memory only, no CUDA call; the paper has no counterpart: it
 * states the problem for a given A, Section 1).  row_ptr (m+1, row_ptr[0] = 0,
 * row_ptr[m] = nnz, non-decreasing), col_idx (nnz, in [0, n)), val (nnz
 * values of `dtype`) -> col_ptr (n+1), row_idx (nnz), val_out (nnz), all
 * caller-owned.  A stable counting sort on the column index: every column's
 * entries come out in increasing row order (entries of one row keep their
 * order), duplicates are kept.  Returns LP_OK, or LP_ERR_ARG for NULL
 * pointers, sizes out of range (n < 2^31) or an invalid CSR structure. */
int lp_csr_to_csc(int32_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                  const void* val, int32_t dtype, int64_t* col_ptr, int32_t* row_idx, void* val_out);

/* Frees the handle and everything it owns.  NULL is accepted. */
int lp_destroy(lp_handle* h);

/* Message of the last error on `h` (empty string if none); valid until the next call. */
const char* lp_last_error(const lp_handle* h);

/* Message of the last lp_create failure on the calling thread (empty after a
 * success); valid until that thread's next lp_create. */
const char* lp_create_error(void);

/* ---- solver ---------------------------------------------------------------- */

/* Runs Algorithm 3 (mode LP_INFEASIBLE) or Algorithm 2 (LP_FEASIBLE) until
 * |c^T x - b^T y|/(1+|c^T x|), ||r_p||/(1+||b||), ||r_d||/(1+||c||) are all <= tol
 * or k_max iterations.  x0, y0, s0 may be NULL: infeasible mode then starts from
 * x0 = s0 = 1, y0 = 0; feasible mode requires a start that is strictly feasible
 * and in N(gamma) (else LP_ERR_NOT_FEASIBLE).  x (n), y (m), s (n) receive the
 * final iterate (NULL to skip).  `io_on_device` applies to x0..s0 and x..s.
 * Returns LP_OK, LP_STATUS_MAX_ITER, LP_STATUS_STALLED or an error; `info`
 * (nullable) receives the summary. */
int lp_solve(lp_handle* h, double tol, int32_t mode,
             const double* x0, const double* y0, const double* s0, int32_t io_on_device,
             double* x, double* y, double* s, lp_result* info);

/* Batched solve of independent LPs (one handle each, created with its own
 * stream: opt.stream = NULL): lp_solve(hs[i], tol, mode, default start, ...)
 * for i < count, run concurrently by up to max_threads host workers (0: one per
 * LP, at most 64), so the kernels of different LPs overlap on the GPU.
 * x, y, s: arrays of count output pointers (entries may be NULL), all host or
 * all device (io_on_device); results: count entries (nullable).  The LPs may
 * have different sizes.  Returns LP_OK when every solve returned a
 * non-negative status (per-LP statuses are in results[i].status), else the
 * first error in index order.  Handles must not be shared between batches
 * running at the same time.  LP_ERR_ARG for hs NULL, count < 0, tol <= 0, a
 * NULL handle or the same handle twice.  If the system refuses to start a
 * host worker, the workers already running (and the calling thread) take its
 * LPs. */
int lp_solve_batch(lp_handle* const* hs, int32_t count, double tol, int32_t mode,
                   int32_t io_on_device, double* const* x, double* const* y, double* const* s,
                   int32_t max_threads, lp_result* results);

/* One inexact normal-equation solve A D^2 A^T dy = p (Algorithm 1 + eq. compv)
 * with the sketch drawn for outer-iteration index k.  D (n) is the diagonal of
 * D; p (m) the right-hand side.  tol_f > 0: stop when ||f^(t)|| <= tol_f;
 * tol_f <= 0: stop when ||f^(t)|| <= tol_cg * ||f^(0)||.  If xs (n, x o s) and
 * v (n) are both non-NULL, v = (XS)^{1/2} W (ADW)^+ (A D^2 A^T dy - p) is
 * returned too (requires D^2 = x/s for the invariant of eq. addl to hold).
 * A draw of W is an embedding only with probability 1 - delta (eq. pdprec):
 * when the Ritz values of the first CG steps spread by more than 1e3 and the
 * solve is still running after 32 steps, W is redrawn (retry + 1, at most
 * twice) and CG continues from the current dy; v uses the final draw.
 * Returns LP_OK, LP_WARN_INNER_MAXIT or an error. */
int lp_normal_solve(lp_handle* h, const double* D, const double* p, const double* xs,
                    int64_t k, double tol_f, int32_t io_on_device,
                    double* dy, double* v, lp_nsolve_info* info);

/* ---- kernel-level entry points (DEVICE pointers; the handle's resident A) ---- */

/* u = A diag(d2) A^T v  (the product inside every CG step, eq. normal).
 * d2 (n), v (m), u (m).  precision 0: products in FP32 with FP32 accumulation
 * (FP32/BF16 storage; FP64 storage always computes in FP64); 1: FP64. */
int lp_adat(lp_handle* h, const double* d2, const double* v, double* u, int32_t precision);

/* Health check of the bounded device-side waits (the paper has no
 * counterpart: this is the failure detection of the GPU pipelines).  Every
 * pipeline wait on an mbarrier gives up after a spin limit (about 1 s),
 * records the timeout in the handle's device status word, waits (again
 * bounded) for its own copies in flight and returns, and the call that
 * launched it returns LP_ERR_DEVICE_TIMEOUT.  This call runs that same wait in
 * one thread on the handle's stream with a spin limit of `spin_cycles`
 * clock64 cycles (1 .. 2^31): with complete = 1 the thread completes the
 * barrier's phase first and the call returns LP_OK; with complete = 0 nothing
 * completes it, so the wait gives up after spin_cycles cycles and the call
 * returns LP_ERR_DEVICE_TIMEOUT.  Nothing else runs and nothing is left in
 * flight; the handle stays usable (every call starts from a clear status
 * word).  LP_ERR_ARG for a NULL handle or arguments out of range. */
int lp_wait_probe(lp_handle* h, int64_t spin_cycles, int32_t complete);

/* Residuals and right-hand side of Algorithm 3 step 3 (Section 5) or eq. pdef:
 * r_p = A x - b (m), r_d = A^T y + s - c (n), mu = x^T s / n, and
 *   infeasible: p = -r_p - sigma mu A S^{-1} 1 + A x - A D^2 r_d
 *   feasible:   p = -sigma mu A S^{-1} 1 + A x.
 * out5 (host, 5 doubles) receives {mu, c^T x, b^T y, ||r_p||, ||r_d||}. */
int lp_residual_rhs(lp_handle* h, const double* x, const double* y, const double* s,
                    int32_t mode, double* r_p, double* r_d, double* p, double* out5);

/* A D W for the CountSketch of (seed, k, retry): adw is m x w, row-major
 * (adw[i*w + j]).  D (n).  Returns the width w through *w_out (nullable). */
int lp_sketch(lp_handle* h, const double* D, uint64_t seed, int64_t k, int32_t retry,
              double* adw, int64_t* w_out);

/* Factors an m x w row-major sketch (QR of its transpose) and keeps the
 * preconditioner in the handle; then z = Q^{-1} r with Q = adw adw^T.
 * Returns LP_ERR_SKETCH_RANK if adw is numerically rank deficient. */
int lp_precond_apply(lp_handle* h, const double* adw, const double* r, double* z);

/* Directions of eqs. (delshat)/(delshat_i) and (delxhat):
 *   ds = -A^T dy (feasible) or -r_d - A^T dy (infeasible);
 *   dx = -x + sigma mu / s - (x/s) o ds - v / s.   rd may be NULL in feasible mode. */
int lp_directions(lp_handle* h, const double* x, const double* s, const double* rd,
                  const double* dy, const double* v, double mu, int32_t mode,
                  double* dx, double* ds);

/* Step lengths of Algorithm 2 steps 5-6 / Algorithm 3 steps 6-7: alpha_max is the
 * first exit from N(gamma) along (dx, ds) in [0, 1] (res_ratio = ||r||/||r^0||
 * and mu0 enter the infeasible condition), alpha_bar minimises the gap on
 * [0, alpha_max].  out2 (host) = {alpha_max, alpha_bar}. */
int lp_step_lengths(lp_handle* h, const double* x, const double* s, const double* dx,
                    const double* ds, int32_t mode, double res_ratio, double mu0,
                    double* out2);

/* Copies up to `max_records` records of the last lp_solve into `recs` (host
 * memory, nullable when max_records == 0); returns the number of records
 * available (>= 0) or LP_ERR_ARG. */
int lp_get_history(lp_handle* h, lp_iter_record* recs, int32_t max_records);

/* ---- checkpoint / resume ----
 * The state of the outer iteration (Algorithm 3, or Algorithm 2 in feasible
 * mode) between two outer steps.  The sketch of outer iteration k is drawn
 * from (seed, k, retry) (Section 6, Algorithm 1 step 1), so a solve resumed
 * from the state taken after k steps draws the same W sequence as the
 * uninterrupted solve and, the rest of the path being deterministic, takes
 * the same iterates.  The neighbourhood of the infeasible method
 * (||r|| / ||r^0|| <= mu / mu_0, Algorithm 3) and the stalling test refer to
 * the start point's mu_0 and ||r^0||, which the state carries along.
 *   k            outer iterations done (the iterate is x_k, y_k, s_k)
 *   mode         LP_FEASIBLE / LP_INFEASIBLE of the solve the state is from
 *   has_dy_prev  1 when dy_prev holds the last outer iteration's dy (kept for
 *                the warm start's "previous" proposal, lp_set_warm_start)
 *   mu0, r0      mu and ||(r_p, r_d)|| at the solve's start point
 *   ratio_ref    the factor check's reference ratio max/min |R_ii| (0: none)
 *   seed         the sketch seed (lp_options.seed) of that solve
 *   mu           mu of the iterate as the solve computed it (by the update's
 *                own reduction, which may differ from x^T s / n summed afresh
 *                in the last bit; the resumed solve takes this value) */
typedef struct {
    int32_t k;
    int32_t mode;
    int32_t has_dy_prev;
    int32_t reserved;  /* 0 */
    double mu0;
    double r0;
    double ratio_ref;
    uint64_t seed;
    double mu;
} lp_state;

/* The state of the last lp_solve on `h` (whatever status >= 0 it returned):
 * `st` (host) and the iterate x (n), y (m), s (n) and dy_prev (m, nullable),
 * host or device buffers by io_on_device.  LP_ERR_ARG when no solve has ended
 * with a status >= 0 since the handle was created, a state was set, or another
 * entry point overwrote the handle's iterate (lp_residual_rhs). */
int lp_get_state(lp_handle* h, lp_state* st, double* x, double* y, double* s, double* dy_prev,
                 int32_t io_on_device);

/* Loads a state (from lp_get_state, on this handle or another one created on
 * the same LP) for the next lp_solve, which then must be called with
 * x0 = y0 = s0 = NULL and the state's mode: it starts at outer iteration
 * st->k from (x, y, s), counts k towards k_max, and takes mu_0, ||r^0||, the
 * factor reference and the sketch seed from the state (the handle's seed is
 * replaced by st->seed).  dy_prev is needed when st->has_dy_prev is 1.
 * LP_ERR_ARG for a null pointer, k < 0, an unknown mode, mu0 <= 0 or
 * mu <= 0, a negative or non-finite r0 or ratio_ref, or reserved != 0. */
int lp_set_state(lp_handle* h, const lp_state* st, const double* x, const double* y,
                 const double* s, const double* dy_prev, int32_t io_on_device);

/* u = A diag(d2) A^T v without any device allocation, for callers that own all
 * device memory themselves (a pre-sized arena, a serving loop with a fixed
 * memory budget, code that must not call the CUDA allocator after start-up)
 * and therefore cannot create a handle.  The paper has no counterpart: this is
 * the FP32 product of the solver's inner loop offered outside a handle.
 *   A   device pointer, column-major, leading dimension ld (elements) with
 *       ld * element size a multiple of 16 bytes, 16-byte aligned, holding
 *       n * ld elements; dtype LP_F32 or LP_BF16.  Rows m .. ld-1 of each
 *       column are padding: they are read but never used, whatever they hold.
 *   d2 (n), v (m), u (m): FP64 device vectors owned by the caller.
 *   stream: cudaStream_t or NULL.
 * The call is synchronous: it returns after the product is done (it reads a
 * status word back and synchronises the stream), so it must not be called
 * while a stream is being captured into a CUDA graph.
 * Scratch lives in one fixed 4 MiB __device__ array inside the library, kept by
 * every device that used it until the library is unloaded; its address is
 * looked up on the first call on each device.  All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  The limit is on the leading dimension,
 * not on m: ld up to 2048 in FP32 and 4096 in BF16 (the kernel's register
 * tile; the fixed array holds the partial sums of any such ld); a larger ld
 * returns LP_ERR_ARG.  Nothing is allocated in any case.  Returns LP_OK, LP_ERR_ARG,
 * LP_ERR_CUDA or LP_ERR_DEVICE_TIMEOUT. */
int lp_adat_noalloc(const void* A, int32_t dtype, int32_t m, int64_t n, int64_t ld,
                    const double* d2, const double* v, double* u, void* stream);

/* Phase-1 primal start (Appendix "Feasible starting point").
 * Rows with b_i < 0 are negated; then the LP
 *     min 1^T z  s.t.  A x + I z = b,  x, z >= 0          (m x (n+m) constraint matrix)
 * is solved by this library's infeasible-start IPM (Algorithm 3, same options)
 * to relative tolerance tol (1e-7 is ample: the start only needs z small next
 * to x, and the phase-1 optimal face is usually unbounded, which makes tight
 * tolerances slow).  A x = b, x >= 0 is feasible exactly when its
 * optimum has z = 0; the interior x > 0 it returns is then moved onto A x = b by
 * the minimum-norm correction x0 = x + A^T (A A^T)^{-1} (b - A x), computed with
 * the sketched normal-equation solver (D = I).
 * A: host matrix (dense column-major, CSC or CSR, any storage dtype; CSR is
 * sorted into CSC first); b: host m-vector;
 * opt: NULL for defaults; x0: caller-owned host n-vector, written when the LP is
 * found feasible.  Returns LP_OK with x0 > 0 and A x0 = b to rounding,
 * LP_ERR_NOT_FEASIBLE when the phase-1 optimum 1^T z exceeds
 * 1e-6 (1 + ||b||) (info->z_sum holds it), LP_ERR_NUMERICAL when the
 * correction leaves some x0_j <= 0, or the error of the inner calls.
 * LP_ERR_ARG, before anything is read or any CUDA call is made: a NULL
 * argument, tol <= 0, a device matrix, m or n < 1, a bad format or dtype, a
 * NULL value array, ld < m (dense), a CSC matrix without pointers or
 * indices, with ptr[0] < 0 or with decreasing column pointers (a row index
 * out of range is found while the phase-1 matrix is built), or a CSR matrix
 * whose structure is not valid. */
typedef struct {
    double z_sum;               /* 1^T z at the phase-1 solution */
    double residual;            /* ||A x0 - b|| after the correction */
    double x0_min;              /* min_j x0_j */
    int32_t outer_iterations;   /* of the phase-1 IPM */
    int64_t inner_total;
} lp_phase1_info;
int lp_phase1_start(const lp_matrix* A, const double* b, const lp_options* opt, double tol,
                    double* x0, lp_phase1_info* info);

/* ---- learned warm start of the inner solve ---------------------------------
 * A multilayer perceptron in -> H -> H -> out with GELU after both hidden layers
 * (trained by mean-squared error with Adam), used to propose the inner solve's
 * starting point.  The paper does not define this; the features are
 *   X = [dy_{k-1} / |u|, u / |u|, log10(mu_k) / 10 * 1_m],  u = Q^{-1} p_k
 * (3m values, dy_{k-1} = 0 at the first outer iteration) and the target is
 * dy_k / |u|, so in = 3m and out = m.  Batches are column-major (features x
 * batch) device FP32 arrays; parameters W1 (H x in), b1, W2 (H x H), b2,
 * W3 (out x H), b3 are column-major in one FP32 vector. */
typedef struct lp_mlp lp_mlp;
int lp_mlp_create(lp_mlp** model, int32_t in, int32_t hidden, int32_t out, uint64_t seed, void* stream);
int lp_mlp_destroy(lp_mlp* model);
int64_t lp_mlp_num_params(const lp_mlp* model);
int lp_mlp_get_params(lp_mlp* model, float* host);       /* host: num_params floats */
int lp_mlp_set_params(lp_mlp* model, const float* host);
int lp_mlp_get_grads(lp_mlp* model, float* host);        /* gradients of the last loss_grad / train_step */
/* Y (out x batch) = model(X (in x batch)), device arrays */
int lp_mlp_forward(lp_mlp* model, const float* X, int32_t batch, float* Y);
/* loss = 1/(2 batch) sum ||model(X) - T||^2 and its gradients (no update) */
int lp_mlp_loss_grad(lp_mlp* model, const float* X, const float* T, int32_t batch, double* loss);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) at learning rate lr on the batch */
int lp_mlp_train_step(lp_mlp* model, const float* X, const float* T, int32_t batch, float lr, double* loss);

/* Warm start of lp_solve's inner solves (fixed-sigma rule).  mode 0: none (the
 * paper: dy^0 = 0); 1: the previous outer iteration's dy; 2: the model's
 * proposal |u| model(X) and the previous dy.  The candidates v_i are combined
 * by one Galerkin step on M = A D^2 A^T, dy^0 = sum c_i v_i with
 * (v_i^T M v_j) c = (v_i^T p) (one FP32 product per candidate), the
 * start of least ||M^{-1} p - dy^0||_M in their span.  dy^0 is used only while
 * mu >= 1e-6 mu_0, only if its true residual is smaller, sqrt(r^T Q^{-1} r) <
 * sqrt(p^T Q^{-1} p) with r = p - M dy^0, and only if |dy^0| <= 4 |Q^{-1} p|;
 * the stopping rule (relative to the cold residual sqrt(p^T Q^{-1} p)) is
 * unchanged, so the iterate returned satisfies the same bound.  Features X
 * (3m, FP32): [dy_{k-1} / |u|, u / |u|, (log10(mu) / 10) 1_m] with
 * u = Q^{-1} p; target dy_k / |u|.  rec_X (3m x capacity) and rec_T
 * (m x capacity), device FP32, nullable: every outer iteration's features and
 * target are appended until capacity (for training).  The model is borrowed,
 * not owned. */
int lp_set_warm_start(lp_handle* h, int32_t mode, lp_mlp* model, float* rec_X, float* rec_T,
                      int32_t rec_capacity);
/* counters since lp_set_warm_start: recorded samples, proposals, accepted proposals */
int lp_get_warm_start_stats(lp_handle* h, int64_t* recorded, int64_t* proposals, int64_t* accepted);

/* Statistics of the hot product kernel (requires opt.profile = 1; the timed
 * launches are the sample described at lp_options.profile). */
int lp_get_kernel_stats(lp_handle* h, lp_kernel_stats* st);

/* Compares every guard region of a handle created with lp_options.guard = 1
 * with its fill pattern (after the handle's stream is idle).  *checked = the
 * number of regions compared (2 per buffer; 0 without the option), *damaged =
 * how many differ; lp_last_error names the first damaged buffer (its index in
 * allocation order and size).  LP_ERR_ARG for null pointers. */
int lp_check_guards(lp_handle* h, int64_t* checked, int64_t* damaged);

/* Device memory of destroyed handles is kept by the library (per device and
 * block size, up to 16 GiB in all) and reused by the next handles, so that
 * creating and destroying handles of one shape again and again (a service
 * solving a stream of LPs) makes no cudaMalloc or cudaFree calls after the
 * first.  A cudaMalloc that fails empties the cache and is retried.  This
 * call returns every cached block to the driver; call it with no handle's
 * work in flight on a block being freed (blocks enter the cache only after
 * their handle's streams were synchronised).  Always LP_OK.  (Not a method
 * of the paper: memory management of the library.) */
int lp_release_cached_memory(void);
int lp_reset_kernel_stats(lp_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* LP_SKETCH_IPM_H */
