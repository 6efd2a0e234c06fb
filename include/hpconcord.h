/*
 * hpconcord.h -- C ABI of a single-GPU (GB300, sm_103a) implementation of the
 * HP-CONCORD proximal-gradient solver for the CONCORD/PseudoNet sparse inverse
 * covariance estimator (Koanantakool et al., arXiv:1710.10769).
 *
 * Problem (Section 2, eq. 1, with the gradient of Alg. 1 step 4): given the
 * observations X (n x p, one observation per row) and lambda1, lambda2 >= 0,
 *
 *   minimise  f(Omega) + lambda1 * sum_{i != j} |w_ij|,
 *   f(Omega) = -sum_i log w_ii + tr(Omega S Omega)/2 + lambda2/2 ||Omega||_F^2,
 *   S = X^T X / n   (no centring),
 *
 * whose smooth-part gradient is G = -diag(1/w_ii) + (S Omega + Omega S)/2 +
 * lambda2 Omega (Alg. 1 step 4).  The solver is Alg. 1: Omega^0 = I; each
 * iteration backtracks over tau = 1, 1/2, 1/4, ... with the soft-threshold
 * prox of eq. (2) applied to the off-diagonal entries, and accepts the first tau
 * passing the sufficient-decrease test of Alg. 1 step 9; it stops when
 * ||Omega^{k+1} - Omega^k||_F / ||Omega^k||_F < eps.  Cov (Alg. 2) forms S once;
 * Obs (Alg. 3) works from X directly.
 *
 * Conventions for every call:
 *  - Dense matrices are row-major.  Pointers are device pointers unless the
 *    argument or option says "host".  The caller owns every buffer it passes;
 *    the library copies what it keeps, so inputs may be freed after the call.
 *  - Work is ordered on the CUDA stream given to hpc_create (NULL = legacy
 *    default stream).  Calls return after the work they enqueue has finished
 *    on that stream, except where stated.
 *  - Every call returns an int status (HPC_OK = 0).  Negative values are
 *    errors; the handle stays usable after HPC_ERR_ARG, HPC_ERR_CAPACITY and
 *    solver errors, and must be destroyed after HPC_ERR_CUDA.
 *  - A handle may be used by one host thread at a time.
 *  - The sparse iterate is symmetric and stored in CSR with both triangles and
 *    the diagonal, columns ascending within each row.
 */
#ifndef HPCONCORD_H
#define HPCONCORD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define HPC_OK                   0
#define HPC_NOT_CONVERGED        1   /* max_iter reached; the iterate is valid            */
#define HPC_ERR_ARG             -1   /* bad argument: lambda < 0, eps <= 0, n/p < 1, NULL */
#define HPC_ERR_OOM             -2   /* device allocation failed                          */
#define HPC_ERR_CAPACITY        -3   /* candidate/iterate capacity exceeded (max_capacity) */
#define HPC_ERR_NONPOS_DIAG     -4   /* a supplied iterate has a diagonal entry <= 0      */
#define HPC_ERR_NAN             -5   /* NaN/Inf met in the gradient or the objective      */
#define HPC_ERR_LS_FAIL         -6   /* no step passed the test within max_halvings       */
#define HPC_ERR_CUDA            -7   /* a CUDA runtime call failed (hpc_last_error())     */
#define HPC_ERR_NOT_IMPLEMENTED -8   /* combination of options not built                  */
#define HPC_ERR_DEVICE_TIMEOUT  -9   /* a bounded device-side wait gave up                */

/* ---------------------------------------------------------------- enums */
typedef struct hpc_ctx* hpc_handle;         /* opaque, owned by the library */

/* Alg. 2 (Cov: S formed once) / Alg. 3 (Obs: Z = Y X / n every iteration);
 * HPC_AUTO picks one at hpc_create by hpc_choose_variant. */
typedef enum { HPC_COV = 0, HPC_OBS = 1, HPC_AUTO = 2 } hpc_variant;

typedef enum { HPC_F32 = 0, HPC_F64 = 1, HPC_BF16 = 2 } hpc_dtype;

/* Arithmetic of the dense products S = X^T X / n (Alg. 2 step 2) and
 * Z = Y X / n (Alg. 3 step 4).  Everything else follows value_dtype.
 * The tensor-core modes sum K in chunks (hpc_tuning.gram_chunk), so their
 * accumulation error does not grow with n: BF16X3 is FP32-class.  For the Obs
 * variant HPC_PREC_FP32 selects that BF16X3 Z product (hpc_get_info then
 * reports HPC_PREC_BF16X3); FP64 and the SIMT modes are Cov only. */
typedef enum {
    HPC_PREC_AUTO   = -1,  /* FP64 for FP64 iterates, BF16X3 otherwise            */
    HPC_PREC_FP64   = 0,   /* SIMT FP64 fused multiply-adds                        */
    HPC_PREC_FP32   = 1,   /* SIMT FP32 fused multiply-adds ("plain FP32")         */
    HPC_PREC_BF16X3 = 2,   /* tensor cores: x = hi + lo in BF16, hi*hi + hi*lo +
                              lo*hi accumulated in FP32; one term when X is BF16  */
    HPC_PREC_TF32   = 3    /* tensor cores, TF32 inputs, FP32 accumulation        */
} hpc_precision;

/* Lemma 3.1's choice between the variants.  With s outer iterations, t line-search
 * trials per iteration and d nonzeros per row of the iterate, Cov costs
 * 2np^2 + 2dp^2(st+1) flops and Obs 2np^2 s + 2dnp(st+1); weighting the dense
 * products (the Gram, Z) by gamma_dense and the sparse-dense work by gamma_sparse
 * (time per flop of each on this GPU), Cov is chosen when
 *   gamma_dense 2np^2 + gamma_sparse 2dp^2(st+1) < gamma_dense 2np^2 s + gamma_sparse 2dnp(st+1).
 * s, t, d and the ratio gamma_sparse / gamma_dense are the arguments; a value <= 0
 * takes the default: s = 40, t = 3, d = 2 and ratio HPC_GAMMA_RATIO.  The ratio is the
 * median measured on GB300 over a sweep of p = 40000, n = 100 ... 12800 on chain and
 * random graphs (gamma_sparse: the Cov iteration's time per flop the lemma counts for
 * it; gamma_dense: the Obs iteration's time per flop of its Z product); it ranged from
 * 12 on the random graph to 121 on the chain, whose noisier S leaves the bound
 * screening less to prune.  With the measured s, t and d of each point the rule picked
 * the faster variant at 14 of the 16 points.  The two modelled costs (in gamma_dense
 * units) go to *cost_cov and *cost_obs (nullable).  Returns HPC_COV or HPC_OBS;
 * HPC_ERR_ARG for n < 1 or p < 1. */
#define HPC_GAMMA_RATIO 26.0
int hpc_choose_variant(int64_t n, int64_t p, double s, double t, double d, double gamma_ratio,
                       double* cost_cov, double* cost_obs);

/* ---------------------------------------------------------------- options / stats */
typedef struct {
    double  eps;            /* stopping tolerance on ||dOmega||_F/||Omega||_F (1e-6)   */
    int64_t max_iter;       /* outer iterations per hpc_solve (1000)                   */
    int32_t max_halvings;   /* tau = 2^-h, h = 0..max_halvings (60)                    */
    int32_t precision;      /* hpc_precision (HPC_PREC_AUTO)                           */
    int32_t value_dtype;    /* HPC_F32 (default) or HPC_F64: S, Omega, G arithmetic    */
    int32_t ls_window;      /* tau values tested per line-search launch, 1..16 (8)     */
    int64_t capacity;       /* initial candidate capacity in entries (0 = 32 p)        */
    int64_t max_capacity;   /* growth limit in entries (0 = p*p)                       */
    int32_t x_on_host;      /* X passed to hpc_create / hpc_load_x is a host pointer.
                               Page-locked (pinned) memory and the tensor-core Gram:
                               the kernels read X where it is, through its device
                               mapping.  Otherwise the handle copies X into a device
                               staging buffer, kept between loads (freed by
                               hpc_destroy).  The host buffer is not used after the
                               call returns.                                          */
    int32_t timing;         /* time the phases into hpc_stats (1): CUDA events around
                               each screening pass, or device timestamps in the device
                               loop                                                    */
    int32_t device_loop;    /* 1 (default): the iteration and line-search loops run on
                               the device, one CUDA-graph launch per solve (conditional
                               WHILE nodes); 0: the host drives every iteration       */
    int32_t reserved_;
} hpc_options;

typedef struct {
    int64_t iterations;       /* outer iterations done by the last call                 */
    int64_t ls_trials;        /* tau values tried (the paper's t summed over iterations) */
    int64_t nnz;              /* entries of the current iterate (both triangles + diag)  */
    int32_t status;           /* same as the call's return value                         */
    int32_t accepted_halvings;/* h of the last accepted tau = 2^-h                       */
    double  f;                /* smooth part f(Omega^k) at the last gradient pass (FP64) */
    double  F;                /* f + lambda1 * sum_{i!=j} |w_ij| at that iterate          */
    double  rel_change;       /* last ||Omega^{k+1}-Omega^k||_F / ||Omega^k||_F          */
    double  ms_total;         /* device time of the call                                 */
    double  ms_gram;          /* device time of the data load: the dense product that
                                 formed S, with its operand transpose and the block
                                 maxima of the bound screening                          */
    double  ms_grad_pass;     /* device time in the gradient-screening pass (Cov SpMM)   */
    int64_t grad_pass_launches;
    int64_t kernel_launches;  /* kernels this library launched during the call           */
    int64_t capacity_regrows; /* times the candidate buffers grew                        */
    int64_t candidates;       /* candidate entries of the last gradient pass             */
    double  ms_gram_kernel;   /* of ms_gram: the tensor-core product kernel alone (without
                                 the transpose of X into its operand panels)             */
} hpc_stats;

/* Fill *opt with the defaults listed above. */
void hpc_default_options(hpc_options* opt);

/* Human-readable text for a status code (static storage). */
const char* hpc_status_string(int status);

/* Text of the last CUDA error seen on this thread ("" if none). */
const char* hpc_last_error(void);

/* ---------------------------------------------------------------- solver handle */

/* Create a solver for X (n x p, dtype xdt, row-major; host pointer when
 * opt->x_on_host) with tuning parameters lambda1, lambda2 >= 0.
 * Cov: computes S = X^T X / n now (Alg. 2 step 2).  Obs: keeps X^T.
 * The iterate starts at Omega = I (Alg. 1 step 1).  cuda_stream is a
 * cudaStream_t (NULL = default stream).  X may be NULL: then call hpc_load_x
 * before solving.  Errors: HPC_ERR_ARG (n,p < 1; lambda < 0; eps <= 0; bad
 * enum; Obs with n > 2097120, the rows its transpose of X takes), HPC_ERR_OOM,
 * HPC_ERR_CUDA, HPC_ERR_NOT_IMPLEMENTED. */
int hpc_create(hpc_handle* out, const void* X, hpc_dtype xdt, int64_t n, int64_t p,
               double lambda1, double lambda2, hpc_variant variant,
               const hpc_options* opt, void* cuda_stream);

/* Replace the data by a new X of the same n, p (host pointer if x_on_host != 0),
 * recompute S (Cov) or X^T (Obs) and reset the iterate to I.  This is the whole
 * set-up cost of a solve: a time-to-converge is hpc_load_x + hpc_solve. */
int hpc_load_x(hpc_handle h, const void* X, hpc_dtype xdt, int x_on_host);

/* Stage the next data set while the handle works on the current one.  The
 * paper's data arrives once per problem (Alg. 1 step 2 builds S from it).  A
 * caller that solves a sequence of data sets can overlap the next one's arrival
 * with the current load and solve.
 *  - Host X is copied into the handle's staging buffer by the copy engine, on a
 *    second stream, starting at once. It needs no SM, so the copy runs alongside
 *    the Gram of the next hpc_load_x. Device X needs no copy.
 *  - That next hpc_load_x (of another X) then queues the staged X's panel
 *    preparation (the tensor-core Gram's transpose) on the second stream, behind
 *    its own Gram, so the preparation overlaps the solve.
 *  - A later hpc_load_x of the staged X (same pointer and type) uses the prepared
 *    panels, or the staged copy if no Gram came in between.
 *  - Pipeline over data sets X_0, X_1, ...: hpc_prefetch_x(X_{k+1}),
 *    hpc_load_x(X_k), hpc_solve, for k = 0, 1, ...  The buffers of consecutive
 *    data sets must differ.
 *  - Arguments as hpc_load_x. X must keep its contents until it has been loaded.
 *  - A load that stages pageable host memory, and hpc_hypergrad, first wait for
 *    the staging and discard it.
 *  - A no-op (HPC_OK) on the other paths (Obs, FP32/FP64 Gram), and before the
 *    first hpc_load_x has sized the handle's buffers. */
int hpc_prefetch_x(hpc_handle h, const void* X, hpc_dtype xdt, int x_on_host);

/* Run Alg. 1 from the current iterate until the stopping rule holds (HPC_OK),
 * max_iter is reached (HPC_NOT_CONVERGED) or an error occurs.  stats may be NULL. */
int hpc_solve(hpc_handle h, hpc_stats* stats);

/* Run exactly k outer iterations from the current iterate, ignoring the stopping
 * rule (for tracing trajectories).  stats may be NULL. */
int hpc_iterate(hpc_handle h, int64_t k, hpc_stats* stats);

/* Copy the current iterate out in CSR.  Call with row_ptr == NULL to query:
 * *nnz_inout receives the entry count.  Otherwise *nnz_inout is the capacity of
 * col/val on entry and the count on return; row_ptr has p+1 entries.  val has
 * dtype vdt (HPC_F32 or HPC_F64).  on_device != 0: all three are device
 * pointers; else host pointers.  HPC_ERR_CAPACITY if the arrays are too short. */
int hpc_get_omega(hpc_handle h, int64_t* nnz_inout, int64_t* row_ptr, int32_t* col,
                  void* val, hpc_dtype vdt, int on_device);

/* Set the iterate (warm start / resume) from a symmetric CSR with a positive
 * diagonal present in every row, columns ascending.  HPC_ERR_NONPOS_DIAG if a
 * diagonal entry is missing or <= 0; HPC_ERR_ARG if not sorted or out of range. */
int hpc_set_omega(hpc_handle h, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                  const void* val, hpc_dtype vdt, int on_device);

/* Change lambda1, lambda2 (>= 0) keeping S and the current iterate (warm start). */
int hpc_set_lambda(hpc_handle h, double lambda1, double lambda2);

/* One point of a regularisation path. */
typedef struct {
    double  lambda1;
    int64_t iterations;       /* outer iterations of this point's solve          */
    int64_t ls_trials;
    int64_t nnz;              /* entries of the estimate (both triangles + diag) */
    int32_t status;           /* HPC_OK, HPC_NOT_CONVERGED or an error           */
    int32_t pad_;
    double  f, F;             /* at the last gradient pass of the solve          */
    double  rel_change;
    double  ms;               /* device time of this point's solve               */
} hpc_path_point;

/* Solve along a grid of lambda1 values at fixed lambda2 -- the grids of tuning
 * parameters that cross-validation and stability selection need (Section 2,
 * "Key bottlenecks") -- in the given order, each solve warm-started from the
 * previous estimate (the first from the current iterate).  Descending lambda1
 * (sparse to dense) keeps warm starts close.  The minimiser is unique for
 * lambda2 > 0, so a warm start changes the path taken, not the estimate.
 * points (host, k entries) receives per-point results.  If row_ptr != NULL the
 * estimates are returned too (host arrays): row_ptr holds k*(p+1) offsets, point
 * t's at row_ptr + t*(p+1), each relative to that point's first entry; col/val
 * (FP32) receive the points' entries back to back, capacity *cap_inout entries,
 * total written on return.  Stops at the first point that returns an error
 * (its status says which); HPC_ERR_CAPACITY if col/val are too short. */
int hpc_solve_path(hpc_handle h, const double* lambda1, int64_t k, double lambda2, hpc_path_point* points,
                   int64_t* row_ptr, int32_t* col, float* val, int64_t* cap_inout);

/* Solve `count` independent problems (handles of the same device) concurrently.
 * When every handle uses the device loop (hpc_options.device_loop, the default)
 * the whole batch is ONE CUDA-graph launch: each handle's iteration loop is an
 * independent branch of the graph, launched on handles[0]'s stream after it
 * waits for the other handles' streams; `threads` is unused.  A handle whose
 * candidate buffers overflow grows them and finishes alone.  Otherwise a pool of
 * at most `threads` host threads (0 = one per stream) drives the handles' solves,
 * so their kernels overlap on the GPU; handles sharing a stream are then solved
 * one after another.  stats (host, count entries, may be NULL) receives each
 * handle's hpc_solve statistics (ms_total: the batch launch's device time).
 * Returns HPC_OK if every solve returned HPC_OK, HPC_NOT_CONVERGED if any stopped
 * at max_iter, and otherwise the first error (by handle index); per-handle
 * statuses are in stats[t].status. */
int hpc_solve_batch(hpc_handle* handles, int count, int threads, hpc_stats* stats);

/* Read m entries S_{rows[t], cols[t]} of the Cov sample covariance into out
 * (FP64, host arrays).  For checking the Gram at sizes where S is too large to
 * copy.  HPC_ERR_ARG for an index outside [0, p) or for the Obs variant. */
int hpc_get_s_entries(hpc_handle h, int64_t m, const int64_t* rows, const int64_t* cols,
                      double* out);

/* Copy out the screened gradient of the last gradient pass: every entry (i, j)
 * that is in the support of the iterate, on the diagonal, or has |G_ij| >
 * lambda1 -- the only entries any prox step can make nonzero (eq. 2) -- with
 * the iterate value w_ij and G_ij (Alg. 1 step 4), as host FP64/int64 arrays.
 * Query with rows == NULL (count into *m_inout).  Entries outside this set
 * satisfy w_ij = 0 and |G_ij| <= lambda1. */
int hpc_get_candidates(hpc_handle h, int64_t* m_inout, int64_t* rows, int64_t* cols,
                       double* omega, double* grad);

/* Resolved configuration of a handle. */
typedef struct {
    int64_t n, p;
    int64_t ld;               /* leading dimension of the stored S (elements)          */
    int32_t variant;          /* hpc_variant                                            */
    int32_t precision;        /* hpc_precision after resolving HPC_PREC_AUTO            */
    int32_t value_dtype;      /* HPC_F32 or HPC_F64                                     */
    int32_t pad_;
    int64_t capacity;         /* current candidate capacity (entries)                   */
    int64_t device_bytes;     /* device memory held by the handle                       */
    double  lambda1, lambda2;
} hpc_info;

/* Fill *info for handle h. */
int hpc_get_info(hpc_handle h, hpc_info* info);

/* ---------------------------------------------------------------- differentiation */

/* Smooth part f(Omega) = -sum log w_ii + tr(Omega S Omega)/2 + lambda2/2 ||Omega||_F^2 at the
 * current iterate (the loss whose gradients hpc_backward returns), into *f (host). */
int hpc_smooth_value(hpc_handle h, double* f);

/* Gradients of L(Omega, X) = f(Omega; S = X^T X / n) at the current (symmetric)
 * iterate, times grad_loss (the upstream derivative of a scalar loss):
 *   dOmega = grad_loss * ( -diag(1/w_ii) + (Omega S + S Omega)/2 + lambda2 Omega )
 *            -- Alg. 1 step 4's G, dense p x ld_domega, bitwise equal to the
 *            solver's G on its candidate entries when grad_loss = 1;
 *   dX     = grad_loss * X Omega^2 / n   (= Y Omega / n with Y = X Omega), n x p.
 * At a non-symmetric Omega the general forms are (Omega^T S + S Omega^T)/2 and
 * (X Omega Omega + X Omega^T Omega^T)/(2n); the iterate is always symmetric.
 * X: the device data (n x p, dtype xdt) the handle was loaded with; needed only
 * for dX.  dOmega, dX: device buffers in the handle's value dtype (FP32, or
 * FP64 for FP64 handles); either may be NULL.  Allocates scratch on first use.
 * HPC_ERR_ARG when dX is asked for with n > 2097120 (the rows of X's transpose). */
int hpc_backward(hpc_handle h, const void* X, hpc_dtype xdt, double grad_loss, void* dOmega, int64_t ld_domega,
                 void* dX);

/* The same gradients with dL/dOmega restricted to the entries of the current
 * iterate: dOmega_vals[e] = grad_loss * G_ij for the e-th entry (i, j) in the
 * order hpc_get_omega returns them (row_ptr / col), FP64 on the device, nnz
 * values; G as in hpc_backward (Alg. 1 step 4), formed without a p x p buffer:
 * (Omega S)_ij from gathers of S (Cov) or from Y^T = Omega X^T and the handle's
 * copy of X^T (Obs).  dX as hpc_backward (Cov only).  Either output may be NULL.
 * Synchronises the handle's stream. */
int hpc_backward_support(hpc_handle h, const void* X, hpc_dtype xdt, double grad_loss, double* dOmega_vals,
                         void* dX);

/* The held-out loss of model selection at the current iterate:
 *   L_val(Omega) = -sum_i log w_ii + tr(Omega S_val Omega) / 2,  S_val = X_val^T X_val / n_val,
 * the unpenalised smooth part of the objective (Section 2, eq. (1) under this library's
 * scaling) on data the estimate was not fitted to.  The paper motivates grids of tuning
 * parameters for cross-validation; this is the criterion evaluated at each point.
 * tr(Omega S_val Omega) = sum over the support of w_ij (Omega S_val)_ij, with
 * (Omega S_val)_ij = <(X_val Omega)_{:,i}, X_val_{:,j}> / n_val: S_val is never formed.
 * Xval: device, nval x p row-major, dtype xdt.  Cov and Obs handles.  Synchronises the
 * handle's stream; the FP64 result goes to *loss (host). */
int hpc_heldout_loss(hpc_handle h, const void* Xval, hpc_dtype xdt, int64_t nval, double* loss);

typedef struct {
    int64_t cg_iterations;
    double  rel_residual;     /* ||r|| / ||b|| of the CG solve                     */
    int64_t support;          /* |A|, entries of the estimate (both triangles)     */
    int32_t converged;        /* rel_residual <= cg_tol reached                    */
    int32_t pad_;
} hpc_hypergrad_info;

/* Gradient of a held-out loss with respect to (lambda1, lambda2) through the
 * fixed point of Alg. 1 (the paper motivates grids of tuning parameters for
 * model selection; this gives their gradient).  With L_val(Omega) = -sum log
 * w_ii + tr(Omega S_val Omega)/2, S_val = X_val^T X_val / n_val (unpenalised),
 * and A the support of the current estimate (held fixed: valid while the
 * support is locally constant in lambda), the implicit function theorem on
 * G_A(Omega) + lambda1 sign_off(Omega_A) = 0 gives
 *   dL_val/dlambda1 = -<v, sign_off(Omega_A)>,  dL_val/dlambda2 = -<v, Omega_A>,
 *   H_A v = grad_A L_val,  H[E] = (E S + S E)/2 + lambda2 E + diag(E_ii / w_ii^2),
 * solved by conjugate gradients (FP64 vectors, relative residual cg_tol, at
 * most cg_max_iter iterations).  Xval: device, nval x p (nval <= 2097120),
 * row-major, caller-owned;
 * S_val is not formed: its term (Omega S_val)_ij on A is read from X_val Omega
 * and X_val (scratch 2 p nval values of the handle's type).  Returns HPC_OK, or
 * HPC_NOT_CONVERGED when cg_max_iter was reached (results still written). */
int hpc_hypergrad(hpc_handle h, const void* Xval, hpc_dtype xdt, int64_t nval, double cg_tol, int64_t cg_max_iter,
                  double* dlambda1, double* dlambda2, hpc_hypergrad_info* info);

/* Free the handle and all device memory it owns.  NULL is accepted. */
int hpc_destroy(hpc_handle h);

/* ---------------------------------------------------------------- stateless products */

/* S = X^T X / n (Alg. 2 step 2) for device X (n x p, dtype xdt, row-major)
 * into device S (p x lds, dtype sdt = HPC_F32 or HPC_F64, lds >= p), both
 * triangles written, S bitwise symmetric.  precision as hpc_precision
 * (HPC_PREC_FP64 needs sdt = HPC_F64).  Enqueued on stream.  The SIMT modes
 * return without synchronising; the tensor-core modes (BF16X3, TF32) allocate
 * stream-ordered scratch for the transposed operand panels and synchronise the
 * stream to check the kernel's error word (HPC_ERR_DEVICE_TIMEOUT if a bounded
 * wait gave up). */
int hpc_gram(const void* X, hpc_dtype xdt, int64_t n, int64_t p, void* S, hpc_dtype sdt,
             int64_t lds, int precision, void* cuda_stream);

/* Allocation-free variant of the tensor-core hpc_gram (the paper has no
 * counterpart: this serves callers of the library, not the method).
 *
 * For callers that must not allocate device memory while they run: code whose
 * device memory belongs to another allocator (for example a framework's caching
 * allocator that has already reserved the budget, so a raw cudaMalloc fails or
 * fragments it), services whose memory budget is fixed at start-up, and
 * latency-critical loops in which cudaMalloc/cudaFree would synchronise the
 * device.  It computes the same S = X^T X / n as hpc_gram with precision
 * HPC_PREC_BF16X3 (also for HPC_PREC_AUTO) or HPC_PREC_TF32, for X of dtype
 * HPC_F32 or HPC_BF16; the caller still passes X and S (device pointers, S is
 * p x lds FP32).  It calls no allocating routine: its scratch is a static
 * 64 MiB device array (HPC_GRAM_NOALLOC_SCRATCH_BYTES) that every GPU loading
 * the library holds until the process exits.
 *
 * Limit: the scratch needed, (panels) * p_pad * n_pad * (2 or 4) bytes plus
 * 8 bytes per tile, with p_pad = p rounded up to 256, n_pad = n rounded up to
 * 64, two BF16 panels for FP32 X in BF16X3, one BF16 panel for BF16 X, one
 * FP32 panel for TF32, must fit in HPC_GRAM_NOALLOC_SCRATCH_BYTES; otherwise
 * the call returns HPC_ERR_ARG and hpc_last_error() states the sizes.
 *
 * The first call on a device looks up the array's device address there (with
 * that device current), so make the first call on each device before any
 * stream capture.  Under CUDA's default lazy module loading that first call is
 * also when the device code is loaded and the 64 MiB array is reserved: a
 * caller with a fixed budget should make it at start-up (or set
 * CUDA_MODULE_LOADING=EAGER, which reserves it when the library is loaded).
 * All calls share the array and it keeps the last call's contents (each call
 * writes everything it reads); calls that overlap on the GPU -- on other
 * streams or from other host threads -- race on it, including on the kernel's
 * error word, which also sits in the array.  The call synchronises the stream
 * before returning (to read that word).  Errors as hpc_gram;
 * HPC_ERR_NOT_IMPLEMENTED (with hpc_last_error() set) if TMA descriptors are
 * unavailable. */
#define HPC_GRAM_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int hpc_gram_noalloc(const void* X, hpc_dtype xdt, int64_t n, int64_t p, float* S, int64_t lds,
                     int precision, void* cuda_stream);

/* ---------------------------------------------------------------- tuning */
/* Launch shapes of a handle's kernels.  The Gram's tiles are summed in the same
 * order whatever their schedule, and the candidates are sorted per row whatever
 * their emission order, so S and the candidate values do not depend on them.
 * The line-search grid (ls_blocks_per_sm) regroups the FP64 partial sums of the
 * sufficient-decrease test, which can move their last bits; a step changes only
 * if that decides an exact tie.  The paper tunes its replication factors and grid
 * shapes per machine (Section 4); these are the single-GPU counterparts.
 * gram_chunk is the exception: it sets how the Gram's FP32 sums are grouped. */
typedef struct {
    int32_t gram_band;         /* row blocks of 128 per band of the tensor-core Gram's
                                  tile order, 1..256 (16): sets which X panels the
                                  tiles running together share in L2               */
    int32_t ls_window;         /* tau values per line-search launch: 1, 2, 4, 8, 16 */
    int32_t ls_blocks_per_sm;  /* resident blocks per SM of the line-search
                                  evaluation, 0 = as many as fit (2)               */
    int32_t rows_ctas_per_sm;  /* CTAs per SM of the off-diagonal row kernel, 1..4 (2);
                                  3 and 4 run a form sized for 3 resident CTAs  */
    int32_t gram_maxima;       /* 1: the tensor-core Gram's epilogue writes the bound
                                  screening's block maxima; 0: a pass over S after it (1) */
    int32_t screen_bounds;     /* 1: the screening pass reads only the segments of S
                                  whose block-maxima bound can emit; 0: it streams the
                                  whole upper triangle and every block of the rows with
                                  neighbours.  Both emit the same entries (1)       */
    int32_t gram_schedule;     /* tensor-core Gram tiles: 1, taken by the persistent
                                  CTAs from a shared counter (the tiles in flight stay
                                  together in the band order); 0, CTA g takes tiles g,
                                  g + grid, ... (1)                                 */
    int32_t gram_chunk;        /* K elements per accumulation chunk of the tensor-core
                                  Gram (and of the Obs Z product), rounded down to a
                                  stage (64 K for BF16 operands, 32 for TF32): each
                                  chunk starts from a zero accumulator and the chunk
                                  sums are added in FP32 round-to-nearest.  Shorter
                                  chunks shrink the bias of the tensor core's
                                  truncating accumulation.  0 = the default (512 for
                                  BF16 X, 256 for BF16X3 and TF32); a value >= n is
                                  one chunk per tile.  It changes S's last bits, so
                                  the autotuner does not touch it (0)               */
    int32_t gram_lead;         /* K elements of each tile's (each Obs pair's) first two
                                  chunks, which keep the tensor core busy while the
                                  epilogue stores the previous tile (emits the previous
                                  pair); 0 = 2 gram_chunk (Gram), 4 gram_chunk (Obs).
                                  Like gram_chunk it groups S's sums: not tuned (0)  */
    int32_t fused_tail;        /* 1: an iteration's steps after the screening pass --
                                  candidate structure, gradient, every line-search
                                  window with its decision, compaction and stopping
                                  rule -- run as one cooperative kernel, grid-wide
                                  barriers between the steps; 0: as the chain of
                                  separate kernels.  The same entries and decisions
                                  either way (the windows' partial sums are grouped
                                  by the line-search grid in both).  On GB300 the two
                                  take the same time to within a few percent (a
                                  barrier costs about a kernel boundary inside the
                                  solve's CUDA graph); the chain is faster where the
                                  candidate structure is large, and where other
                                  streams run kernels during the solve (a cooperative
                                  kernel waits until its whole grid is resident: it
                                  queues behind hpc_prefetch_x's transpose).  Not
                                  touched by the autotuner.  hpc_solve_batch's single
                                  graph launch runs its problems' loops concurrently,
                                  always on the chain; handles solved from its worker
                                  threads keep their own setting (0)               */
} hpc_tuning;

/* The bound screening's block maxima of the Cov variant: out[i * nb + jb] = max
 * |S_ij| over the column block jb (columns 128 jb .. 128 jb + 127, 64 in FP64 mode)
 * with j != i and j < p, rounded up to BF16 (bit patterns), nb = ceil(p / block).
 * The tensor-core Gram writes them from its epilogue; the other modes by a pass
 * over S.  Query with out == NULL (p * nb into *count_inout); HPC_ERR_CAPACITY if
 * *count_inout is smaller; HPC_ERR_NOT_IMPLEMENTED for the Obs variant. */
int hpc_get_block_maxima(hpc_handle h, int64_t* count_inout, uint16_t* out);

/* Read / replace a handle's tuning.  HPC_ERR_ARG for a value out of range. */
int hpc_get_tuning(hpc_handle h, hpc_tuning* t);
int hpc_set_tuning(hpc_handle h, const hpc_tuning* t);

#define HPC_TUNE_MAX_TRIALS 48
typedef struct {
    int32_t knob;              /* 0 gram_band, 1 ls_window, 2 ls_blocks_per_sm,
                                  3 rows_ctas_per_sm, 4 gram_maxima, 5 gram_schedule */
    int32_t value;
    double  ms;                /* Gram knobs: one data load (transpose, product, block
                                  maxima); the others: one iteration                */
} hpc_tune_trial;

typedef struct {
    int32_t ntrials;
    int32_t pad_;
    hpc_tune_trial trials[HPC_TUNE_MAX_TRIALS];
} hpc_tune_report;

/* The autotuner: times the candidate values of each knob on the handle's own
 * problem and keeps the fastest, one knob after another.
 *  - If X != NULL (same conventions as hpc_load_x) the whole load is timed for
 *    each gram_band candidate, then for gram_maxima 1 and 0: three round-robin
 *    rounds over the candidates, each keeping its fastest load (the SM clock
 *    drifts under the power cap).  S is rewritten with identical values.
 *  - The iteration knobs (ls_window, rows_ctas_per_sm, ls_blocks_per_sm) are
 *    timed over `iters` outer iterations (>= 1) each,
 *    every trial starting from the handle's current iterate, which is restored
 *    afterwards: the call leaves the estimate unchanged.  Start from a
 *    representative iterate (for example after a few hpc_iterate calls) for
 *    timings that reflect a solve.
 * The chosen tuning is applied to the handle and written to *best (nullable);
 * every trial is listed in *report (nullable).  Times are CUDA events on the
 * handle's stream.  Errors as hpc_iterate / hpc_load_x. */
int hpc_autotune(hpc_handle h, const void* X, hpc_dtype xdt, int x_on_host, int64_t iters, hpc_tuning* best,
                 hpc_tune_report* report);

#ifdef __cplusplus
}
#endif
#endif /* HPCONCORD_H */
