/*
 * gpsparse.h -- C ABI of the GB300 sparse exact-GP library.
 *
 * The library evaluates the exact Gaussian process of arXiv 2205.09070
 * (Noack, Krishnan, Risser, Reyes, "Exact Gaussian Processes for Massive
 * Datasets via Non-Stationary Sparsity-Discovering Kernels") on one GPU:
 *
 *   K = A * k~(|x_i - x_j| ; r_s) * sum_m f_m(x_i) f_m(x_j) + sigma_n^2 I
 *       (Sec. 2.2, Eq. eq:bump_kernel with the stationary kernel of
 *        Eq. eq:kstat; f_m is the bump sum of Eq. eq:bump)
 *   ln L = -1/2 y^T K^-1 y - 1/2 ln|K|          (Sec. 2.1, Eq. eqn:log_likelihood)
 *
 * K is assembled as a sparse CSR matrix (cell-list pair search, count, scan,
 * fill); y^T K^-1 y comes from conjugate gradients and ln|K| from stochastic
 * Lanczos quadrature on the same CG iterations (Sec. 2.5 solves K x = y by
 * CG and estimates the log-determinant by randomized linear algebra).
 *
 * Conventions shared by every entry point
 *  - Points x: N x dim doubles, row-major (x[i*dim + k]).  Targets y: N doubles.
 *  - Array arguments may be HOST or DEVICE pointers; the library detects which
 *    (cudaPointerGetAttributes) and copies host data itself.  The caller owns
 *    every array it passes; the library never keeps a caller pointer beyond
 *    the call.
 *  - Hyperparameters h: host array of gp_n_params() doubles laid out as
 *      for m < n_funcs, b < n_bumps: [centre (dim), radius r_mb, amplitude a_mb]
 *      then r_s (stationary support radius), A (stationary amplitude),
 *      sigma_n^2 (noise variance), and with GP_CORE_SQEXP the core length
 *      scale l.
 *    This is the hyperparameter set of Eq. eq:bump / eq:kstat; the bump shape
 *    beta is a fixed constant of the context (Sec. 3 counts 42 parameters for
 *    n_funcs = 2, n_bumps = 4, dim = 3: no beta among them).
 *  - The prior mean is zero and the additive constant -N/2 ln(2 pi) is
 *    dropped, as in Eq. eqn:log_likelihood.
 *  - Every call is ordered on the context's CUDA stream.  Calls that return
 *    host scalars synchronise that stream before returning.
 *  - Return value: GP_OK (0) or one of the GP_ERR_* codes; no C++ exception
 *    crosses this boundary and no kernel traps.  On an error, outputs are
 *    unspecified unless stated otherwise.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef GPSPARSE_H
#define GPSPARSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GP_OK                 0
#define GP_ERR_INVALID_ARG    1  /* bad size, null pointer, non-finite or out-of-range h, non-finite y */
#define GP_ERR_CUDA           2  /* a CUDA runtime call failed */
#define GP_ERR_OOM            3  /* device allocation failed */
#define GP_ERR_NOT_CONVERGED  4  /* CG hit max_iter before every column met cg_rtol; outputs are filled */
#define GP_ERR_NOT_SPD        5  /* CG breakdown: p^T K p <= 0 or not finite (K not positive definite) */
#define GP_ERR_TIMEOUT        6  /* a bounded device-side wait gave up */
#define GP_ERR_NOT_ASSEMBLED  7  /* gp_solve / gp_get_csr before a successful gp_assemble */
#define GP_ERR_UNSUPPORTED    8  /* a size above a compiled limit (dim > 3, n_funcs > 32, ...) */

/* arithmetic of the path */
#define GP_FP64        0  /* coordinates, kernel values, vectors and scalars in FP64; single-RHS CG */
#define GP_FP32_MIXED  1  /* FP32 kernel values, CSR and CG vectors (batched [y, probes]);
                             FP64 dot products, CG scalars, Lanczos eigensolve and log-det sums;
                             FP64 re-check of every support test inside a guard band */

typedef struct gp_ctx gp_ctx; /* opaque: owns the CSR matrix and all device workspaces */

/* Core kernel k_c multiplying the sparsity-discovering kernel (Sec. 2.2: any
 * kernel k_c may be combined as k_c * k_s; the paper's figure shows a squared
 * exponential core):
 *   GP_CORE_NONE   K = A k~ sum_m f_m f_m + sigma_n^2 I
 *   GP_CORE_SQEXP  K = A k~ exp(-|x_i - x_j|^2 / (2 l^2)) sum_m f_m f_m + sigma_n^2 I,
 *                  with the length scale l > 0 one more hyperparameter, the
 *                  last entry of h.  k_c(x, x) = 1, so the diagonal, the
 *                  pattern and the sparsity bound do not depend on l. */
#define GP_CORE_NONE  0
#define GP_CORE_SQEXP 1

/* Kernel family (Eq. eq:bump_kernel): dim in 1..3, n_funcs (n1) in 1..32,
 * n_bumps (n2) >= 1 with n_funcs*n_bumps <= 512, beta > 0 (shape of every
 * bump), core one of GP_CORE_*. */
typedef struct {
  int32_t dim;
  int32_t n_funcs;
  int32_t n_bumps;
  double beta;
  int32_t core;
} gp_kernel_desc;

typedef struct {
  int32_t precision;      /* GP_FP64 or GP_FP32_MIXED */
  int32_t n_probes;       /* Rademacher probes for SLQ / Hutchinson, 1..64 */
  int32_t lanczos_steps;  /* Lanczos (CG) steps used by SLQ, 1..64; with GP_FLAG_LOGDET_TAYLOR
                             the number of series terms, 1..4096 */
  int32_t max_iter;       /* CG iteration cap */
  double cg_rtol;         /* stop a column when |r| <= cg_rtol |r0| (Jacobi-scaled system) */
  uint64_t seed;          /* probe stream: SplitMix64 counter l*2^40 + original point index */
  int32_t check_every;    /* iterations between host convergence checks (0: default 16) */
  int32_t flags;          /* GP_FLAG_* bits */
  int32_t precond_block;  /* FP32_MIXED only: 0 = Jacobi scaling alone; 8, 16, 32, 64 or 128 = also
                             block-Jacobi preconditioned CG, blocks of that many consecutive
                             rows of the Morton-ordered active block (see gp_lml) */
  int32_t batch_workers;  /* gp_lml_grad_batched: host threads that run the instances' assembly
                             and gradient (grouped CG launches), or whole instances on as many
                             worker streams, each with its own workspace (0: automatic,
                             min(n_inst, 8); at most 16) */
} gp_opts;

/* gp_opts.flags: time every launch of the SpMM, pair-fill and adjoint kernels
 * with CUDA events on the context stream (reported in gp_info.t_*_kernel_ms). */
#define GP_FLAG_TIME_KERNELS 1
/* gp_opts.flags: run the FP32 path's sparse product Q = K P (one per CG
 * iteration) in the given form instead of the autotuner's choice.  Without
 * these bits the first FP32 solve of each matrix shape (n_active, block count,
 * columns) in the process times every form on that matrix (4 launches each,
 * one host synchronisation) and keeps the fastest for the life of the process;
 * contexts then agree on the form for a given shape.  The forms give the same
 * products summed in different orders (FP32 rounding differences only). */
#define GP_FLAG_SPMM_CPASYNC  2  /* stage filled by per-lane cp.async copies */
#define GP_FLAG_SPMM_TMA      4  /* stage filled by TMA: tile::gather4 of P rows, bulk copy of values */
#define GP_FLAG_SPMM_TMA_WIDE 8  /* TMA stage, 2 or 3 float4 columns per lane (else as GP_FLAG_SPMM_TMA) */
#define GP_FLAG_SPMM_CPASYNC_WIDE 32  /* cp.async stage, 2 or 3 float4 columns per lane (else as
                                         GP_FLAG_SPMM_CPASYNC) */
#define GP_FLAG_SPMM_WINDOW 64  /* column windows: tiles of 8 block rows stream the union of their
                                   columns through a shared-memory ring filled by TMA bulk copies
                                   (one persistent CTA per SM); the product also forms the CG step */

/* gp_opts.flags: estimate ln|K| with the randomized estimator the paper cites
 * (Sec. 2.5, Boutsidis et al.) instead of stochastic Lanczos quadrature: on
 * the same Jacobi-scaled active block and probes,
 *   ln|Khat| ~ mean_l [N_act ln a - sum_{k=1}^{m} z_l^T C^k z_l / k],
 *   C = I - Khat / a,  a = max_i sum_j |Khat_ij| (Gershgorin, >= lambda_max),
 * with m = lanczos_steps terms (one SpMM over the probe block per term).  The
 * series converges like (1 - lambda_min / a)^m, so for ill-conditioned K it
 * is biased low at any practical m; gp_info.logdet_stderr reports the
 * spread over probes only.  FP32_MIXED only (else GP_ERR_UNSUPPORTED); the
 * gradient's trace term is Hutchinson's on the same probes either way. */
#define GP_FLAG_LOGDET_TAYLOR 16

/* gp_opts.flags: failure injection for tests of the error paths, all made on
 * the host (no device fault, trap or hang):
 *   GP_FLAG_FAULT_OOM     every device allocation the call needs fails as an
 *                         out-of-memory would (GP_ERR_OOM); buffers the context
 *                         already holds are kept
 *   GP_FLAG_FAULT_NOT_SPD gp_lml / gp_lml_grad negate the assembled matrix
 *                         before the solve, so CG meets p^T K p < 0
 *                         (GP_ERR_NOT_SPD)
 *   GP_FLAG_FAULT_NAN     gp_lml / gp_lml_grad write a NaN into one stored
 *                         entry before the solve, so the CG scalars turn
 *                         non-finite (GP_ERR_NOT_SPD)
 * The next call without the flags re-assembles and runs normally. */
#define GP_FLAG_FAULT_OOM 128
#define GP_FLAG_FAULT_NOT_SPD 256
#define GP_FLAG_FAULT_NAN 512

/* gp_opts.flags: gp_lml_grad_batched runs every instance on its own on the
 * worker streams, even where its grouped CG launches apply (see there). */
#define GP_FLAG_BATCH_STREAMS 1024

/* gp_info.spmm_variant */
#define GP_SPMM_CPASYNC  0
#define GP_SPMM_TMA      1
#define GP_SPMM_TMA_WIDE 2
#define GP_SPMM_CPASYNC_WIDE 3
#define GP_SPMM_WINDOW 4

typedef struct {
  int64_t n;              /* points */
  int64_t n_active;       /* points inside the support of some bump (rows that couple) */
  int64_t nnz;            /* stored entries of the active block (diagonal included) */
  int32_t iters;          /* CG iterations run (max over columns / solves) */
  int32_t status_detail;  /* column that failed, or -1 */
  double max_rel_resid;   /* largest recursive relative residual at exit */
  double quad_form;       /* y^T K^-1 y */
  double logdet;          /* estimated ln|K| */
  double logdet_stderr;   /* standard error of the SLQ mean over probes (x N_active) */
  double t_assemble_ms;
  double t_solve_ms;
  double t_grad_ms;
  double cell_size;       /* edge of the uniform search grid */
  int64_t n_cells;        /* cells in the search grid */
  int64_t launches;       /* kernels this call launched (no-op CG launches after convergence included) */
  int32_t n_spmm;         /* SpMM launches that did work (GP_FLAG_TIME_KERNELS) */
  int32_t kp;             /* padded RHS columns of the batched CG */
  double t_spmm_kernel_ms;    /* summed device time of those SpMM launches */
  double t_fill_kernel_ms;    /* device time of the pair-fill kernel */
  double t_adjoint_kernel_ms; /* device time of the adjoint pair kernel */
  int32_t lanczos_iters;  /* iterations of the separate SLQ Lanczos run (preconditioned
                             evaluations only, else 0) */
  int32_t precond_block;  /* block size the solve used (0: none) */
  int32_t spmm_variant;   /* GP_SPMM_* form of the FP32 sparse product, -1 if none ran */
} gp_info;

/* Number of hyperparameters: n_funcs*n_bumps*(dim+2) + 3, plus 1 with GP_CORE_SQEXP. */
int64_t gp_n_params(const gp_kernel_desc* desc);

/* Sparsity bound of Sec. 2.2 (Eq. eq:sparsity_estimate and the two equations
 * after it): for uniformly distributed points the fraction of non-zero
 * covariances is at most
 *   s(h) = sum_i sum_j sum_k Vol(dim, r_ij) Vol(dim, r_ik) / domain_volume^2,
 *   Vol(dim, r) = pi^(dim/2) / Gamma(dim/2 + 1) r^dim,
 * over the bump radii r_ij of h (layout as for gp_assemble).  Writes s and,
 * if grad is not NULL, d s / d h (gp_n_params doubles; only the radius
 * entries are non-zero).  Host arrays; no device work.  GP_ERR_INVALID_ARG
 * for a non-positive or non-finite radius or domain volume. */
int gp_sparsity_estimate(const gp_kernel_desc* desc, const double* h, double domain_volume, double* s,
                         double* grad);

/* Augmented objective of Sec. 2.4 (Eq. eq:augmented) exactly as printed:
 * ln L + (1 - s) ln L = (2 - s(h)) ln L(h), with s the sparsity bound of
 * gp_sparsity_estimate, and its gradient by the product rule,
 * (2 - s) d ln L / d h - ln L d s / d h.  Two properties a caller should know:
 *  - s is the uncapped upper bound of Sec. 2.2; it exceeds 1 when the bumps'
 *    balls overlap enough (it is a bound, not a fraction), and for s > 2 the
 *    weight (2 - s) on ln L changes sign;
 *  - d value / d s = -ln L, so for ln L < 0 (the usual case) a larger s (a
 *    denser K) raises the value: the objective favours sparsity only where
 *    ln L > 0.
 * lml and lml_grad are what gp_lml_grad returned for h; grad (gp_n_params
 * doubles) may be NULL, and then lml_grad may be NULL too.  s_out (may be
 * NULL) receives s(h), which is also what a caller compares with its sparsity
 * requirement for the constrained form (Eq. eq:constrained).  Host arrays; no
 * device work. */
int gp_augmented(const gp_kernel_desc* desc, const double* h, double domain_volume, double lml,
                 const double* lml_grad, double* value, double* grad, double* s_out);

/* gp_train objectives (Sec. 2.4; the paper names gradient-based training as
 * future work, Sec. 4):
 *   GP_OBJ_LML          ln L(h)
 *   GP_OBJ_AUGMENTED    (2 - s(h)) ln L(h), Eq. eq:augmented (gp_augmented)
 *   GP_OBJ_CONSTRAINED  ln L(h) subject to s(h) < s_max, Eq. eq:constrained */
#define GP_OBJ_LML 0
#define GP_OBJ_AUGMENTED 1
#define GP_OBJ_CONSTRAINED 2

typedef struct {
  int32_t objective;      /* GP_OBJ_* */
  int32_t n_steps;        /* ascent steps, 0..100000 (each needs one gp_lml_grad evaluation) */
  double lr;              /* Adam step size (> 0) in the parametrisation of gp_train */
  double beta1, beta2;    /* Adam moment decays in [0, 1) (0, 0: 0.9, 0.999) */
  double eps;             /* Adam denominator guard (> 0; 0: 1e-8) */
  double domain_volume;   /* V of the sparsity estimate s(h) (gp_sparsity_estimate), > 0 */
  double s_max;           /* GP_OBJ_CONSTRAINED: the sparsity requirement; s(h) < s_max at the start */
  int32_t max_halvings;   /* GP_OBJ_CONSTRAINED: halvings of a step that would reach s >= s_max
                             before the step is skipped (0: 30) */
} gp_train_opts;

/* Gradient ascent on an objective of the hyperparameters h (gp_n_params
 * doubles, host, updated in place) for the data x, y (as gp_lml_grad), with
 * Adam (Kingma and Ba, 2015) on theta: theta_q = ln h_q for the entries that
 * must stay positive (bump radii, r_s, A, sigma_n^2 and the core length
 * scale; A must then start > 0), theta_q = h_q for centres and amplitudes, so
 * d obj / d theta_q = h_q d obj / d h_q for the former.  Step t (1-based):
 *   g = d obj / d theta at h_{t-1} (ln L and its gradient from gp_lml_grad
 *       with opts, s and its gradient from gp_sparsity_estimate),
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   theta += lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * GP_OBJ_CONSTRAINED keeps every iterate feasible: a step that would reach
 * s >= s_max is halved until s < s_max, and skipped after max_halvings
 * halvings (s depends on the radii alone, so this needs no evaluation).
 * trace (may be NULL): (n_steps + 1) rows of 3 doubles, (objective, ln L, s)
 * at h_0 .. h_{n_steps}; info (may be NULL) describes the last evaluation.
 * Errors: GP_ERR_INVALID_ARG for bad options, a non-positive A, or an
 * infeasible start; an evaluation's error (GP_ERR_NOT_CONVERGED included)
 * stops the run and is returned, with h the iterate it was evaluated at and
 * the trace filled up to the row before it. */
int gp_train(gp_ctx* ctx, const double* x, const double* y, int64_t n, double* h, const gp_opts* opts,
             const gp_train_opts* train, double* trace, gp_info* info);

/* Default options: FP32_MIXED, 32 probes, 50 Lanczos steps, 10000 iterations,
 * rtol 1e-6, seed 0x5eed, check every 16 iterations, precond_block 128. */
void gp_default_opts(gp_opts* opts);

/* Create a context on CUDA device `device`, ordered on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  The context allocates
 * device memory lazily and keeps it (grow-only) until gp_destroy. */
int gp_create(gp_ctx** out, const gp_kernel_desc* desc, int device, void* cuda_stream);
int gp_destroy(gp_ctx* ctx);
/* Change the stream later calls are ordered on. */
int gp_set_stream(gp_ctx* ctx, void* cuda_stream);

/* Assemble K for points x (N x dim) and hyperparameters h (Sec. 2.2,
 * Eq. eq:bump_kernel): bump table, active-point compaction, Morton-sorted
 * cell list with edge >= r_s, per-row pair count, prefix scan, fill.
 * Uses opts->precision only.  Synchronises the stream once (to size the CSR).
 * N may be 0.  The matrix stays in the context until the next assemble. */
int gp_assemble(gp_ctx* ctx, const double* x, int64_t n, const double* h,
                const gp_opts* opts, gp_info* info);

/* Copy the assembled active block out (diagnostics and tests).
 * Internal row order is the Morton order of the active points; perm[r] is the
 * original index of internal row r; columns are internal indices, ascending
 * within a row; values are unscaled K entries (doubles) whatever the precision.
 * Pass NULL arrays to query the sizes only: sizes[0] = n_active, sizes[1] = nnz.
 * Arrays: row_ptr n_active+1, col nnz, val nnz, perm n_active (host or device). */
int gp_get_csr(gp_ctx* ctx, int64_t* row_ptr, int32_t* col, double* val,
               int32_t* perm, int64_t sizes[2]);

/* Copy-out that allocates no device memory.  No counterpart in the paper.
 * For callers that must not call cudaMalloc at this point: a process whose
 * device memory is entirely handed out by another allocator (a serving
 * runtime's memory pool), or one already at its device-memory limit, still
 * needs the assembled matrix, and gp_get_csr would grow a context buffer for
 * the unscaled values.  Same outputs and conventions as gp_get_csr, but the
 * unscaled values are staged in a fixed area of static device memory inside
 * the library (GP_NOALLOC_MAX_NNZ doubles, 8 MiB, held by every device that
 * loads the library until the process exits) instead of a context buffer.
 *  - If val is not NULL and nnz > GP_NOALLOC_MAX_NNZ: returns
 *    GP_ERR_UNSUPPORTED and copies nothing (use gp_get_csr).
 *  - The first call on a device looks up the staging area's device address
 *    (cudaGetSymbolAddress, with that device current): make that first call
 *    before any stream capture starts.
 *  - Every call shares the staging area, which keeps the last call's values;
 *    each call overwrites every entry it copies out, so nothing needs
 *    clearing.  Two calls whose GPU work overlaps (different streams or host
 *    threads on the same device) race on the area: order them on one stream.
 *  - Synchronises the context stream before returning, so the context stream
 *    must not be a stream that is being captured into a CUDA graph. */
#define GP_NOALLOC_MAX_NNZ (1 << 20)
int gp_get_csr_noalloc(gp_ctx* ctx, int64_t* row_ptr, int32_t* col, double* val,
                       int32_t* perm, int64_t sizes[2]);

/* Solve K alpha = y with the last assembled K (Sec. 2.5: CG; block-Jacobi
 * preconditioned when opts->precond_block > 0 and K is FP32).  Rows outside
 * every bump decouple: alpha_i = y_i / sigma_n^2 there.  alpha: N doubles. */
int gp_solve(gp_ctx* ctx, const double* y, double* alpha, const gp_opts* opts, gp_info* info);

/* Posterior mean at test points (Sec. 2.1: m(x*) = kappa^T (K + V)^-1 y with
 * kappa_i = k(x*, x_i) from Eq. eq:bump_kernel and zero prior mean; V =
 * sigma_n^2 I is part of K).  Solves K alpha = y with the last assembled K
 * exactly as gp_solve does (same opts), then for every test point sums
 * k(x*, x_i) alpha_i over the training points within r_s of it that share the
 * support of some f_m with it (a cell-list pass over the assembled grid, FP64
 * throughout; no noise term, a test point is not an observation).
 *   y:     N doubles (the training targets of the assembled points)
 *   xstar: n_star x dim doubles, row-major; any coordinates (points outside the
 *          training box or every bump get mean 0 where no pair is in support)
 *   mean:  n_star doubles
 * Arrays may be host or device.  Returns GP_ERR_NOT_ASSEMBLED before a
 * gp_assemble, GP_ERR_NOT_CONVERGED (means still written) if CG hit max_iter.
 * info (may be NULL) reports the solve as gp_solve does. */
int gp_predict(gp_ctx* ctx, const double* y, const double* xstar, int64_t n_star, double* mean,
               const gp_opts* opts, gp_info* info);

/* Posterior variance at test points (Sec. 2.1, Eq. eq:pred_distr: the
 * posterior covariance at x* is k(x*, x*) - kappa^T (K + V)^-1 kappa with
 * kappa_i = k(x*, x_i); V = sigma_n^2 I is part of K; this is the variance of
 * the latent function, with no noise term).  With the last assembled K, the
 * test points are taken in blocks of 64; each block's kappa columns, Jacobi-
 * scaled, are solved together as one right-hand-side block of the same CG
 * (block-Jacobi preconditioned in FP32 when opts ask for it, single-column FP64
 * CG otherwise), and var_q = k(x*_q, x*_q) - kappa_q^T K^-1 kappa_q with a
 * compensated sum.  k(x*, x*) = A C sum_m f_m(x*)^2, so points outside every
 * bump get variance 0.
 *   xstar: n_star x dim doubles, row-major;  var: n_star doubles
 * Arrays may be host or device.  GP_ERR_NOT_ASSEMBLED before a gp_assemble;
 * GP_ERR_NOT_CONVERGED (variances still written) if a block's CG hit
 * max_iter.  info (may be NULL) reports the largest iteration count. */
int gp_predict_var(gp_ctx* ctx, const double* xstar, int64_t n_star, double* var, const gp_opts* opts,
                   gp_info* info);

/* Assemble K and evaluate ln L (Eq. eqn:log_likelihood) with
 * ln|K| = sum ln D + SLQ(D^-1/2 K D^-1/2) + N_inactive ln sigma_n^2, D = diag K.
 * The estimator does not depend on precond_block.  With B = precond_block > 0
 * (FP32_MIXED) the SLQ coefficients come from a run of lanczos_steps plain CG
 * (Lanczos) iterations on [yhat, z], and the solves Khat u = [yhat, z] that the
 * quadratic form and the gradient need run as preconditioned CG with
 * M = blockdiag(Khat over consecutive B-row blocks of the Morton-ordered
 * active rows), which converges in far fewer iterations. */
int gp_lml(gp_ctx* ctx, const double* x, const double* y, int64_t n, const double* h,
           const gp_opts* opts, double* lml, gp_info* info);

/* As gp_lml, plus d ln L / d h (host array of gp_n_params doubles):
 * 1/2 alpha^T K_h alpha - 1/2 tr(K^-1 K_h), the trace by Hutchinson's
 * estimator on the same probes, K_h recomputed on the CSR pattern and never
 * stored (the paper lists gradient-based training as future work, Sec. 4). */
int gp_lml_grad(gp_ctx* ctx, const double* x, const double* y, int64_t n, const double* h,
                const gp_opts* opts, double* lml, double* grad, gp_info* info);

/* Many independent GPs that share the kernel family.  Instance k owns points
 * offsets[k] .. offsets[k+1]-1 of x / y (offsets: host, n_inst+1 entries) and
 * hyperparameters h[k*P .. (k+1)*P).  lml: n_inst doubles, grad: n_inst*P
 * doubles (host or device); grad may be NULL.  info (may be NULL) gets totals
 * (iters: the largest instance's count).  Workspaces are kept in ctx for later
 * calls; the work starts after what is already queued on the context stream,
 * and the call returns when all instances are done.
 *
 * Grouped CG launches (the default for FP32_MIXED with the SLQ estimator):
 * instances are taken largest first in waves of up to 256, one workspace and
 * stream each.  opts->batch_workers host threads assemble them; then the CG
 * iterations of all of them run as single launches on the context stream,
 * each launch doing one iteration for every instance still running (an
 * instance leaves when its run finishes); then the threads form each
 * instance's ln L and gradient.  The product is the wide cp.async form (else
 * the cp.async form) for every instance, and each instance's result is the one
 * gp_lml_grad gives for it alone with GP_FLAG_SPMM_CPASYNC_WIDE set (the same
 * kernels and grid, the same reduction order).
 *
 * Worker streams (GP_FLAG_BATCH_STREAMS, FP64, GP_FLAG_LOGDET_TAYLOR, the
 * fault flags, or another GP_FLAG_SPMM_* form): opts->batch_workers workers
 * each take whole instances, largest first, on their own stream, and each
 * instance's result is the one gp_lml_grad gives for it alone with the same
 * options. */
int gp_lml_grad_batched(gp_ctx* ctx, int32_t n_inst, const int64_t* offsets,
                        const double* x, const double* y, const double* h,
                        const gp_opts* opts, double* lml, double* grad, gp_info* info);

const char* gp_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* GPSPARSE_H */
