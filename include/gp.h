/*
 * gp.h -- C ABI of libgp.so: on-the-fly Gaussian-process kernel products and the
 * GP training loss on one GB300 (sm_103a).
 *
 * Problem statement (HiGP, arXiv 2503.02259, §Gaussian Processes): training points
 * X in R^{n x d}, observations y in R^n, test points X* in R^{m x d}, and
 * hyper-parameters Theta = (s, f, l): noise s, scale f, length-scale l.  The
 * regularised kernel matrix is read as
 *
 *     Kh = f^2 K_l + s I,     K_l[i][j] = k(|x_i - x_j|; l),
 *
 * with k the Gaussian kernel exp(-r^2/(2 l^2)) or the Matern-3/2 kernel
 * (1 + sqrt(3) r/l) exp(-sqrt(3) r/l).  Kh is never stored: every product
 * evaluates kernel tiles on the fly and discards them (§Statement of Need).
 *
 * Conventions shared by every call
 *  - Memory: arrays named X, V, Y, B, Xsol, y, alpha, Xstar, mu, Z and probes
 *    are DEVICE pointers (cudaMalloc'ed or from a device tensor) of float32,
 *    row-major, densely packed (leading dimension = number of columns).
 *    Scalar outputs (loss, grad, iters, relres, logdet, info) are HOST pointers.
 *  - Ownership: the caller owns every buffer.  No call allocates device memory;
 *    calls that need scratch take a caller-provided workspace `ws` of at least
 *    gp_workspace_bytes(op, ...) bytes, 256-byte aligned.  The workspace is
 *    scratch only: its contents on entry are ignored.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  gp_kernel_matmul, gp_kernel_grad_matmul, gp_predict_mean and
 *    gp_generate_probes are asynchronous on `stream`.  Calls with host scalar
 *    outputs synchronise `stream` before returning.
 *  - Errors: every call returns a gp_status; no exceptions cross the ABI.
 *    Outputs are valid only on GP_OK, except that iters/relres are also written
 *    on GP_ERR_NOT_CONVERGED.  gp_last_error() returns a thread-local message
 *    describing the last non-OK status of the calling thread.
 *  - Argument checks (GP_ERR_ARG): n >= 1, 1 <= d <= GP_MAX_DIM,
 *    1 <= w <= GP_MAX_COLS, s > 0, f > 0, l > 0, non-NULL device pointers,
 *    kernel in {GAUSSIAN, MATERN32}.
 *  - Statelessness (§Design and Implementation: the interfaces are stateless):
 *    no call keeps state between calls except the thread-local error string,
 *    per-device launch-configuration caches, and one private stream per host
 *    thread and device on which the solvers capture their CG-iteration graphs.
 *  - CG step: after each product the O(n w) part of a CG iteration (alpha,
 *    the x / r update, beta and the stopping test, the p update) runs as one
 *    cooperative launch with two grid barriers (bounded: a barrier that waits
 *    more than 4 s returns GP_ERR_TIMEOUT).  The environment variable
 *    GP_CG_FUSED=0 selects three separate launches instead; both give the same
 *    bits.  The request server's workers always use the separate launches.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GP_MAX_DIM 16     /* largest supported point dimension d */
#define GP_MAX_COLS 128   /* largest multivector width w per product */
#define GP_MAX_LANCZOS 64 /* largest number of Lanczos steps k for SLQ */
#define GP_MAX_PRECOND_RANK 4096 /* largest rank of the Nystrom preconditioner */

typedef enum {
  GP_OK = 0,
  GP_ERR_ARG = 1,            /* invalid argument (message in gp_last_error) */
  GP_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed */
  GP_ERR_OOM = 3,            /* workspace too small / server admission refused */
  GP_ERR_NOT_CONVERGED = 4,  /* CG hit cg_maxit before cg_rtol */
  GP_ERR_BREAKDOWN = 5,      /* CG breakdown: p^T Kh p <= 0 or non-finite */
  GP_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  GP_ERR_UNIMPLEMENTED = 7,  /* combination not built (e.g. precision/kernel) */
  GP_ERR_NUMERIC = 8         /* non-finite or non-positive Lanczos eigenvalue */
} gp_status;

typedef enum { GP_KERNEL_GAUSSIAN = 0, GP_KERNEL_MATERN32 = 1 } gp_kernel;

/* Arithmetic of the K-tile x V-tile contraction.
 *  FP32:   CUDA-core FP32 FMA.
 *  TF32:   tcgen05 tensor cores, kernel tile and V rounded to TF32, FP32
 *          accumulation in tensor memory (about 3e-4 relative).
 *  BF16:   kernel tile rounded to BF16, V as a BF16 high part plus a BF16
 *          remainder (two products; a few 1e-3 relative).
 *  TF32X3, BF16X3: both operands split into a high part and a rounded
 *          remainder, accumulating hi*hi + hi*lo + lo*hi (FP32-level accuracy).
 * Tensor-core accumulation restarts every 512 columns j and is summed in FP32.
 * The tensor-core modes need w <= 128. */
typedef enum {
  GP_PREC_FP32 = 0,
  GP_PREC_TF32 = 1,
  GP_PREC_BF16 = 2,
  GP_PREC_TF32X3 = 3,
  GP_PREC_BF16X3 = 4
} gp_precision;

typedef enum {
  GP_OP_MATMUL = 0,       /* gp_kernel_matmul */
  GP_OP_GRAD_MATMUL = 1,  /* gp_kernel_grad_matmul */
  GP_OP_PCG = 2,          /* gp_pcg_solve */
  GP_OP_SLQ = 3,          /* gp_slq_logdet */
  GP_OP_LOSS_GRAD = 4,    /* gp_loss_and_grad, gp_nll_forward, gp_nll_backward */
  GP_OP_PREDICT = 5,      /* gp_predict_mean */
  GP_OP_RESIDUAL = 6,     /* gp_true_residual, gp_residual_rows */
  GP_OP_PREDICT_VAR = 7,  /* gp_predict_var */
  GP_OP_LOSS_GRAD_BATCH = 8, /* one member of gp_loss_and_grad_batch */
  GP_OP_NYSTROM = 9          /* gp_nystrom_apply */
} gp_op;

/* Theta = (s, f, l): noise s, scale f, length-scale l (§Gaussian Processes). */
typedef struct {
  double s, f, l;
} gp_theta;

/* X: device, n x d row-major float32 training points. kernel: a gp_kernel.
 * ls: optional HOST array of d per-dimension length-scales l_1..l_d (the
 * "kernel parameters l" of §Gaussian Processes taken one per coordinate;
 * theta.l is then unused but must still be > 0), or NULL for the isotropic
 * theta.l.  The kernel sees rho^2 = sum_t (x_t - y_t)^2 / l_t^2:
 * exp(-rho^2/2) or (1 + sqrt(3) rho) exp(-sqrt(3) rho).  Per-dimension
 * length-scales are taken by the products (but not by the dKh/dl output of
 * gp_kernel_grad_matmul), CG, SLQ, the loss and its gradient (which then has
 * 2 + d entries), and the predictions; iterative refinement and the residual
 * calls return GP_ERR_UNIMPLEMENTED for them, as does the request server,
 * whose requests carry no ls. */
typedef struct {
  const float* X;
  int64_t n;
  int32_t d;
  int32_t kernel;
  gp_theta theta;
  const double* ls;
} gp_problem;

/* Options of the iterative solvers.
 *  nprobe:     Rademacher probes p for SLQ and Hutchinson (0 <= p < GP_MAX_COLS).
 *  nlanczos:   Lanczos steps k per probe (1 <= k <= GP_MAX_LANCZOS).
 *  cg_maxit:   CG iteration cap (<= 0: n).
 *  cg_rtol:    per-column stop at ||b - Kh x||_2 / ||b||_2 <= cg_rtol (recurrence
 *              residual, FP64 norms).
 *  refine_rtol: outer tolerance of mixed-precision iterative refinement (used
 *              when prec != FP32; <= 0 disables refinement).
 *  seed:       probe seed; probe (row i, column c) = +1 if the top bit of
 *              SplitMix64(seed ^ (c << 40) ^ i) is 0, else -1.
 *  prec:       contraction precision of the inner products (gp_precision).
 *  probes:     optional device n x nprobe float32 probe block; NULL = generated
 *              from `seed` by the rule above.
 *  refine_maxit: cap on outer refinement steps (<= 0: 10).
 *  slq_prec:   arithmetic of the SLQ Lanczos products (gp_slq_logdet,
 *              gp_loss_and_grad, gp_nll_forward): a gp_precision, or
 *              GP_PREC_SAME for `prec`.  Zero-initialised options run SLQ in
 *              FP32.  The log-determinant of a smooth, ill-conditioned K-hat
 *              needs kernel entries to about 24 bits (FP32 or TF32X3), while
 *              the CG solves tolerate BF16X3, so the two may differ.
 *  refine_residual: arithmetic of the refinement's outer residual
 *              (gp_residual_arith; zero-initialised options select the
 *              compensated FP32-pair form).
 *  precond_rank: 0 = no preconditioner (M = I); k in [1, GP_MAX_PRECOND_RANK]
 *              = the Nystrom preconditioner M = s I + L L^T with L the
 *              rank-k pivoted partial Cholesky factor of f^2 K (see
 *              gp_nystrom_apply), used by gp_pcg_solve,
 *              gp_pcg_solve_refined (in the refinement's inner solves) and
 *              gp_loss_and_grad (Eq. 1 / Eq. 2 with this M); the other calls
 *              reject it (GP_ERR_UNIMPLEMENTED).
 *  precond_tol: the factor stops before k columns once the largest residual
 *              diagonal is <= precond_tol * f^2 (<= 0: only when it is <= 0). */
typedef struct {
  int32_t nprobe;
  int32_t nlanczos;
  int32_t cg_maxit;
  int32_t prec;
  double cg_rtol;
  double refine_rtol;
  uint64_t seed;
  const float* probes;
  int32_t refine_maxit;
  int32_t slq_prec;
  int32_t refine_residual;
  int32_t precond_rank;
  double precond_tol;
} gp_solve_opts;

/* slq_prec value meaning "the same arithmetic as prec". */
#define GP_PREC_SAME (-1)

/* Arithmetic of the O(n^2 w) sums of a residual B - Kh X (X in FP64).
 *  PAIR: FP32-pair ("double-float") arithmetic on the FP32 pipe: exact
 *        differences of the FP32 points, kernel entries by a table-driven pair
 *        exponential (Tang's method) and pair square root, pair products and
 *        compensated sums; about 1e-14 relative per kernel entry.
 *  FP64: FP64 kernel entries and sums (GB300's FP64 pipe is far slower; kept
 *        as the checker). */
typedef enum { GP_RESIDUAL_PAIR = 0, GP_RESIDUAL_FP64 = 1 } gp_residual_arith;

/* Diagnostics of one loss/gradient evaluation (host struct, filled on GP_OK). */
typedef struct {
  double yalpha;           /* y^T Kh^-1 y */
  double logdet;           /* SLQ estimate of log|Kh| (Eq. 1, M = I) */
  double logdet_stderr;    /* standard error of the probe mean */
  double quad[3];          /* alpha^T dKh/dtheta alpha, theta = s, f, l */
  double trace[3];         /* Hutchinson tr(Kh^-1 dKh/dtheta) (Eq. 2, M = I) */
  double trace_stderr[3];
  int32_t cg_iters;        /* largest CG iteration count over the columns */
  int32_t refine_steps;    /* outer refinement steps taken (0 for FP32) */
  double relres_y;         /* final recurrence relres of the y column */
  double relres_max;       /* largest final relres over all columns */
  double logdet_m;         /* log|M| of the preconditioner (0 for M = I; included in logdet) */
  double trace_m[3];       /* tr(M^-1 dM/dtheta) (0 for M = I; included in trace) */
} gp_loss_info;

/* Library version string (static storage). */
const char* gp_version(void);
/* Thread-local message of the calling thread's last non-OK status ("" if none). */
const char* gp_last_error(void);
/* Static name of a status code. */
const char* gp_status_string(gp_status st);

/* Workspace bytes needed by `op` for this problem.  w is the multivector width
 * for MATMUL / GRAD_MATMUL / PCG (ignored otherwise); opts may be NULL for the
 * matmul ops.  For PREDICT, w is the number of test points m.  Returns 0 on an
 * invalid argument (see gp_last_error). */
size_t gp_workspace_bytes(gp_op op, const gp_problem* prob, int32_t w, const gp_solve_opts* opts);

/* Y = Kh V  (the on-the-fly MatVec, §Statement of Need).
 * V, Y: device n x w float32 (may not alias).  prec selects the contraction
 * arithmetic.  Asynchronous on `stream`. */
gp_status gp_kernel_matmul(const gp_problem* prob, const float* V, int32_t w, float* Y,
                           int32_t prec, void* ws, size_t ws_bytes, void* stream);

/* Y = Kh V exactly like gp_kernel_matmul with FP32 arithmetic, but without any
 * device allocation and without a caller workspace.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory at the point of the call -- for example a plug-in running
 * inside a host application (an inference server, another framework's
 * custom-op hook) that owns the device allocator and forbids cudaMalloc in
 * its execute callback, or a fixed-budget loop that must not allocate once it
 * has started.  They still own V and Y.
 *  - Scratch: a file-scope static device array of GP_NOALLOC_SCRATCH_BYTES
 *    (32 MiB), which every GPU that loads the library keeps until the process
 *    exits.  Problems whose scratch (staged points, padded V and the partial
 *    sums of the product) does not fit are rejected with GP_ERR_ARG and a
 *    message giving the bytes needed; the product is first re-planned with
 *    fewer j-splits to fit.  At one split about n * (d_pad + 2 * w_pad) * 4
 *    bytes are needed (d_pad = 2 for d <= 2, else d rounded up to a multiple
 *    of 4; w_pad >= w, a multiple of 4), so n can reach about 120,000 at
 *    d = 3, w = 32.
 *  - Set-up: the first call on each device (with that device current) looks
 *    up the array's device address once; make that first call before any
 *    stream capture.
 *  - Sharing: every call on a device uses the same array, which keeps the
 *    previous call's contents (each call clears what must start at zero).
 *    Calls whose work overlaps on the GPU (different streams or host threads
 *    without ordering) race on the array; order them.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine.
 *    Asynchronous on `stream`. */
#define GP_NOALLOC_SCRATCH_BYTES (32u << 20)
gp_status gp_kernel_matmul_noalloc(const gp_problem* prob, const float* V, int32_t w, float* Y,
                                   void* stream);

/* Fused product of Kh and its derivatives with one multivector, sharing one
 * distance/kernel evaluation per entry (the "kernel matrices and its
 * derivatives" of §Design and Implementation):
 *   Y = Kh V,  dY_f = (dKh/df) V = 2 f K V,  dY_l = (dKh/dl) V = f^2 D_l V,
 * and (dKh/ds) V = V, which is not written.  dY_f or dY_l may be NULL to skip.
 * Asynchronous on `stream`. */
gp_status gp_kernel_grad_matmul(const gp_problem* prob, const float* V, int32_t w, float* Y,
                                float* dY_f, float* dY_l, int32_t prec, void* ws,
                                size_t ws_bytes, void* stream);

/* Column-wise CG for Kh Xsol = B from Xsol = 0 (PCG of §Gaussian Processes; M = I,
 * or the Nystrom preconditioner when opts->precond_rank > 0).  B, Xsol: device n x w.  iters[w], relres[w]: host outputs (iterations
 * and final recurrence relres per column).  Stops each column at opts->cg_rtol
 * or opts->cg_maxit.  With opts->prec != FP32 and refine_rtol > 0 the inner
 * products run on tensor cores and an outer FP32-compensated residual loop
 * refines Xsol until ||B - Kh Xsol|| / ||B|| <= refine_rtol per column.
 * Returns GP_ERR_NOT_CONVERGED (with iters/relres/Xsol written) if a column
 * misses its tolerance.  Synchronises `stream`. */
gp_status gp_pcg_solve(const gp_problem* prob, const float* B, int32_t w, float* Xsol,
                       const gp_solve_opts* opts, int32_t* iters, double* relres, void* ws,
                       size_t ws_bytes, void* stream);

/* True relative residual of a solution: relres[c] = ||B_c - Kh X_c||_2 / ||B_c||_2
 * for each column c < w, with FP64 kernel entries and FP64 sums (the checker
 * of the refinement's residual), e.g. to check the FP32 solution of
 * gp_pcg_solve.  B, X: device n x w float32; relres[w]: host.  Workspace:
 * gp_workspace_bytes(GP_OP_RESIDUAL, prob, w, NULL).  O(n^2 w) FP64 work.
 * Synchronises. */
gp_status gp_true_residual(const gp_problem* prob, const float* B, const float* X, int32_t w,
                           double* relres, void* ws, size_t ws_bytes, void* stream);

/* Residual rows of an FP64 solution: R[k][c] = B[r_k][c] - (Kh X64)[r_k][c]
 * for k < m, c < w, where r_k = rows[k] (rows: device int64 array of m
 * indices in [0, n)) or r_k = k when rows is NULL; the sum over all n points
 * in the arithmetic `arith` (gp_residual_arith).  This is the outer residual
 * of mixed-precision iterative refinement (§Gaussian Processes, PCG; the
 * paper's own arithmetic is FP32), exposed so that a caller can measure it
 * on all rows or on sampled rows.  B: device n x w float32; X64: device
 * n x w float64; R: device m x w float64 (may be NULL); relres: host [w]
 * (may be NULL, not both), ||R_c||_2 / ||B_{rows,c}||_2.  1 <= m <= n.
 * Workspace: gp_workspace_bytes(GP_OP_RESIDUAL, prob, w, NULL) serves any m.
 * GP_ERR_ARG if a row index is out of range (R then holds NaN in that row).
 * Synchronises. */
gp_status gp_residual_rows(const gp_problem* prob, const float* B, const double* X64, int32_t w,
                           const int64_t* rows, int64_t m, int32_t arith, double* R,
                           double* relres, void* ws, size_t ws_bytes, void* stream);

/* Mixed-precision iterative refinement of Kh Xsol = B with an FP64 solution
 * (PCG of §Gaussian Processes, refined; M = I, or the Nystrom preconditioner
 * in the inner solves when opts->precond_rank > 0, built once per call).  Outer loop: R = B - Kh X
 * with X held in FP64 and the sums in the arithmetic opts->refine_residual
 * (default: compensated FP32 pairs; the kernel entries never leave the FP32
 * pipe); inner loop: block CG on the product of precision opts->prec (a
 * tensor-core mode, or FP32) for Kh D = R to opts->cg_rtol, then X += D; stop
 * each column at ||R|| / ||B|| <= opts->refine_rtol or after
 * opts->refine_maxit outer steps.  B: device n x w float32; X64: device n x w
 * float64 (returning the refined solution in FP32 would cost about
 * u ||Kh|| ||X|| / ||B|| of residual).  iters[w]: total inner CG iterations;
 * relres[w]: final outer relative residual.  Workspace:
 * gp_workspace_bytes(GP_OP_PCG, prob, w, opts) with opts->refine_rtol > 0.
 * Synchronises. */
gp_status gp_pcg_solve_refined(const gp_problem* prob, const float* B, int32_t w, double* X64,
                               const gp_solve_opts* opts, int32_t* iters, double* relres, void* ws,
                               size_t ws_bytes, void* stream);

/* Nystrom preconditioner of Kh (the preconditioner M of the PCG in §Gaussian
 * Processes; the paper's own M, AFN, also builds a Nystrom factor on chosen
 * landmark points).  Builds L, the partial Cholesky factor of f^2 K with
 * greedy diagonal pivoting: step j takes the pivot p_j = argmax_i d_i of the
 * residual diagonal d = diag(f^2 K - L L^T) (the smallest index among equal
 * values; the first pivot is 0) and sets
 *   L[:, j] = (f^2 K[:, p_j] - L[:, :j] L[p_j, :j]^T) / sqrt(d_{p_j}),
 * stopping after k columns or once the largest d_i is <= tol * f^2; then
 * applies M^-1 = (s I + L L^T)^-1 to V by the Woodbury identity,
 *   Z = (V - L C^-1 L^T V) / s,  C = s I + L^T L  (C^-1 formed in FP64).
 * L is stored in FP32; its column dot products, L^T L, L^T V and L (C^-1 L^T V)
 * are summed with exact products and FP32-pair sums, so Z is M^-1 V for the
 * stored L up to the final rounding to FP32.  With per-dimension length-scales
 * the points are divided by l_t in FP32 first.
 * k: 1 <= k <= GP_MAX_PRECOND_RANK (k > n is taken as n).  V, Z: device n x w
 * float32 (w >= 1; may not alias).  L (may be NULL): device float32, column j
 * at L + j * n (n rows; columns >= *rank untouched).  piv (may be NULL): host
 * int64 [k], pivots of the built columns.  rank: host, columns built.
 * Workspace: gp_workspace_bytes(GP_OP_NYSTROM, prob, w, opts) with
 * opts->precond_rank = k.  GP_ERR_NUMERIC if C's FP64 Cholesky factorisation
 * meets a non-positive pivot.  Synchronises. */
gp_status gp_nystrom_apply(const gp_problem* prob, int32_t k, double tol, const float* V, int32_t w,
                           float* Z, float* L, int64_t* piv, int32_t* rank, void* ws,
                           size_t ws_bytes, void* stream);

/* SLQ estimate of log|Kh| (Eq. 1 with M = I; stochastic Lanczos quadrature):
 * k steps of Lanczos with full reorthogonalisation from q_1 = z_i / ||z_i||
 * for each probe z_i (FP64 coefficients, products in opts->slq_prec), the
 * tridiagonal T_k eigen-decomposed on the device in FP64 (implicit QR), and
 * logdet = (1/p) sum_i ||z_i||^2 sum_j U_1j^2 log(lambda_j).
 * logdet_stderr = sample std / sqrt(p).  Synchronises `stream`. */
gp_status gp_slq_logdet(const gp_problem* prob, const gp_solve_opts* opts, double* logdet,
                        double* logdet_stderr, void* ws, size_t ws_bytes, void* stream);

/* L(Theta) = 1/2 (y^T Kh^-1 y + log|Kh| + n log 2 pi) and dL/d(s, f, l) =
 * 1/2 (-alpha^T dKh alpha + tr(Kh^-1 dKh))   (§Gaussian Processes: the NLL and
 * gradient equations; Eq. 1 and Eq. 2 with M = I).  One block CG on [y | Z],
 * SLQ from the probe columns, and one fused derivative product with [alpha | Z].
 * y: device n float32.  loss, grad[3] (s, f, l), info (may be NULL): host.
 * With per-dimension length-scales (prob->ls) grad has 2 + d entries
 * (s, f, l_1..l_d), from one fused contraction of the kernel entries and
 * their d derivatives with alpha alpha^T and U Z^T / p (no derivative
 * product is formed); 1 + nprobe <= 48 then, info->quad/trace hold s and f
 * in [0..1] and NaN in [2], and no trace standard errors are formed.
 * With opts->precond_rank > 0 (isotropic l only) the terms of Eq. 1 and
 * Eq. 2 are taken with the Nystrom preconditioner M = s I + L L^T, its pivots
 * held fixed for the derivatives:
 *   log|Kh| = log|M| + log|M^-1/2 Kh M^-1/2|, log|M| = (n - r) log s + log|C|
 *   (C = s I + L^T L), the second term by SLQ on M^-1/2 Kh M^-1/2 (Lanczos in
 *   the M-inner product, weight z^T M^-1 z);
 *   tr(Kh^-1 dKh) = tr(M^-1 dM) + tr(Kh^-1 dKh - M^-1 dM): the first in closed
 *   form ((n - r)/s + tr(C^-1), (2/f)(r - s tr(C^-1)), 2 tr(C^-1 L^T dL/dl),
 *   with dL/dl the forward derivative of the factor's column steps), the
 *   second by the Hutchinson terms (Kh^-1 z)^T dKh (M^-1 z) - (M^-1 z)^T dM (M^-1 z);
 * with probes z = L e1 + sqrt(s) e2 ~ N(0, M) for standard normal e1, e2:
 * opts->probes, if given, is then a device (n + precond_rank) x nprobe
 * float32 row-major block holding e2 in rows [0, n) and e1 in the rows after
 * (only the first r of those are used), else e is generated from opts->seed
 * (Box-Muller on the probe hash with bit 39 of the key set).  The CG solves
 * run preconditioned.  info->logdet_m and info->trace_m give the closed-form
 * terms.  Synchronises `stream`. */
gp_status gp_loss_and_grad(const gp_problem* prob, const float* y, const gp_solve_opts* opts,
                           double* loss, double* grad, gp_loss_info* info, void* ws,
                           size_t ws_bytes, void* stream);

/* gp_loss_and_grad for `count` independent problems at once (1 <= count <=
 * 64): the members advance together, and every CG iteration, every Lanczos
 * step and the gradient pass run ONE grouped product launch covering all
 * members' tiles (a persistent kernel whose CTAs take (member, row tile,
 * j-split) work items from a counter, largest members first), followed by
 * each member's O(n w) steps.  Each member's results are those of its own
 * problem; a member that has converged skips its tiles on the device.  The
 * members share the kernel, the dimension template (d in {1}, {2}, {3}, {4},
 * {5..8}, {9..16}), nprobe (1 + nprobe <= 64) and nlanczos; each has its own
 * X, n, Theta, y, seed, cg_rtol and cg_maxit; products are FP32 and the
 * length-scale isotropic (GP_ERR_UNIMPLEMENTED otherwise).  probs, y (device
 * pointers), opts, ws, ws_bytes: arrays of count; ws[k] of at least
 * gp_workspace_bytes(GP_OP_LOSS_GRAD_BATCH, &probs[k], 0, &opts[k]) bytes.
 * loss[count], grad[3 count], info[count] (may be NULL), status[count] (may
 * be NULL): host.  Returns GP_ERR_NOT_CONVERGED if a member missed its
 * cg_rtol (its results are written, as for gp_loss_and_grad), else the first
 * other error.  Synchronises `stream`. */
gp_status gp_loss_and_grad_batch(int32_t count, const gp_problem* probs, const float* const* y,
                                 const gp_solve_opts* opts, double* loss, double* grad,
                                 gp_loss_info* info, int32_t* status, void* const* ws,
                                 const size_t* ws_bytes, void* stream);

/* The forward half of gp_loss_and_grad: block CG on [y | Z] and SLQ.  Writes the
 * solutions W = Kh^-1 [y | Z] to the device n x (1 + nprobe) array `W` (kept by
 * the caller for the backward half) and the loss.  Synchronises `stream`. */
gp_status gp_nll_forward(const gp_problem* prob, const float* y, const gp_solve_opts* opts,
                         float* W, double* loss, gp_loss_info* info, void* ws,
                         size_t ws_bytes, void* stream);

/* The backward half: from W of gp_nll_forward (same problem, same opts, so the
 * same probes Z are regenerated rather than stored), one fused derivative
 * product with [alpha | Z] gives grad[3] = dL/d(s, f, l) (grad[2 + d] with
 * per-dimension length-scales, as for gp_loss_and_grad).  Synchronises. */
gp_status gp_nll_backward(const gp_problem* prob, const gp_solve_opts* opts, const float* W,
                          double* grad, gp_loss_info* info, void* ws, size_t ws_bytes,
                          void* stream);

/* Posterior mean mu = f^2 K(Xstar, X) alpha at m test points (noise-free test
 * outputs, §Gaussian Processes; the prediction call of §Design and
 * Implementation).  alpha: device n; Xstar: device m x d; mu: device m.
 * prec must be a valid gp_precision, but the product always runs in FP32 on
 * the CUDA cores: one column (w = 1) is far too narrow for a tensor-core tile.
 * Workspace: gp_workspace_bytes(GP_OP_PREDICT, prob, m, NULL).  Asynchronous. */
gp_status gp_predict_mean(const gp_problem* prob, const float* alpha, const float* Xstar,
                          int64_t m, float* mu, int32_t prec, void* ws, size_t ws_bytes,
                          void* stream);

/* Posterior variance of the noise-free test outputs at m test points
 * (§Gaussian Processes: y* and y jointly Gaussian with Cov(y*) = f^2 K(X*, X*),
 * Cov(y, y*) = f^2 K(X, X*), Cov(y) = Kh; the prediction call of §Design and
 * Implementation):  var[c] = f^2 - k_c^T Kh^-1 k_c,  k_c = f^2 K(X, x*_c).
 * Test points are taken in blocks of up to GP_MAX_COLS: the block's columns
 * k_c are formed on the device, Kh^-1 k_c by block CG (opts->cg_rtol,
 * opts->cg_maxit, product arithmetic opts->prec), and the dot products in FP64.
 * In exact arithmetic a CG iterate from zero underestimates k_c^T Kh^-1 k_c,
 * so an unconverged solve overestimates the variance; the FP32 rounding of the
 * difference (about kappa u f^2) can dominate where the variance is far below
 * f^2 on a very ill-conditioned system, and can then even make it negative.  Xstar: device m x d; var: device m
 * float32.  iters_max / relres_max (host, may be NULL): the largest CG
 * iteration count and final relres over all columns.  GP_ERR_NOT_CONVERGED
 * (var written) if a column missed cg_rtol.  Workspace:
 * gp_workspace_bytes(GP_OP_PREDICT_VAR, prob, m, opts).  Synchronises. */
gp_status gp_predict_var(const gp_problem* prob, const float* Xstar, int64_t m, float* var,
                         const gp_solve_opts* opts, int32_t* iters_max, double* relres_max,
                         void* ws, size_t ws_bytes, void* stream);

/* Z[i][c] = +-1 (the probe rule of gp_solve_opts.seed) for i < n, c < p, into the
 * device array Z with leading dimension ldz >= p.  Asynchronous. */
gp_status gp_generate_probes(int64_t n, int32_t p, uint64_t seed, float* Z, int64_t ldz,
                             void* stream);

/* ---------------------------------------------------------------------------
 * Measurement hooks (no counterpart in the paper; used by the benchmark).
 * Between gp_profile_begin and gp_profile_end on one host thread, the library
 * records a CUDA event pair around every launch of the dominant on-the-fly
 * product kernel on the caller's stream, and counts every kernel it launches.
 * gp_profile_end synchronises those events and returns the summed device time
 * of the product kernels (ms), their launch count and the total launch count.
 * At most 65536 product launches are timed per window.
 * ------------------------------------------------------------------------- */
gp_status gp_profile_begin(void);
gp_status gp_profile_end(double* product_ms, int64_t* product_launches, int64_t* total_launches);

/* Pipe-rate microbenchmarks of the current device (no counterpart in the
 * paper): the FP32 FMA pipe driven by packed FP32x2 FMAs (TFLOP/s, an FMA = 2
 * flops) and the MUFU ex2 rate (10^9 ex2 per second), each from one timed
 * launch of about 20 ms on `stream` after one untimed launch.  These are the
 * pipes that bound the on-the-fly product (the contraction and the kernel
 * evaluation).  Allocates nothing; synchronises.  GP_ERR_ARG for NULL
 * outputs, GP_ERR_CUDA if a launch fails. */
gp_status gp_measure_pipe_rates(double* fp32_tflops, double* mufu_ex2_gops, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request server on one device (the stateless
 * loss/gradient and prediction calls of §Design and Implementation, served as
 * a stream of requests; the paper has no server).
 *  - gp_server_create reserves one device pool of hbm_budget_bytes and starts
 *    max_slots worker threads, each with one CUDA stream per stream-priority
 *    level of the device; a request runs on the stream whose priority falls
 *    with its work (entries x columns), so small requests are not queued
 *    behind the tiles of large ones.
 *  - gp_server_submit copies the request's HOST arrays into staging (a pinned
 *    host pool reserved at creation, 1/8 of the budget between 64 MiB and
 *    2 GiB; pageable memory when it is full) and queues it; a request whose
 *    footprint (inputs + outputs + solver workspace) exceeds the whole budget
 *    is refused with GP_ERR_OOM.
 *  - Admission: when a worker is free, the queued request with the least work
 *    (entries x columns) among those whose footprint fits the pool's free
 *    space starts; a request that has waited 30 s or more starts before any
 *    younger one, in arrival order (it waits for room if it does not fit), so
 *    large requests are not starved.  Requests that arrive while others run
 *    join them on the device; their kernels overlap through the workers'
 *    streams.
 *  - Kind 0 runs gp_loss_and_grad; kind 1 solves alpha = Kh^-1 y by block CG and
 *    returns the posterior mean at Xstar.  With a fixed CG budget (cg_maxit) a
 *    result may carry GP_ERR_NOT_CONVERGED with its estimates filled in.
 *  - Results do not depend on what else runs: every kernel is deterministic.
 * ------------------------------------------------------------------------- */
typedef struct gp_server gp_server;

typedef struct {
  int64_t submitted, completed, refused;
  int64_t peak_active;     /* most requests on the device at once */
  size_t peak_bytes;       /* most pool bytes in use at once */
  size_t budget_bytes;
  int64_t batches;         /* grouped launches of two or more requests */
  int64_t batched_requests;/* requests that ran in them */
  int64_t largest_batch;
} gp_server_stats;

typedef struct {
  int32_t kind;            /* 0 = loss + gradient, 1 = posterior-mean prediction */
  int32_t d;
  int64_t n;
  int32_t kernel;
  int32_t nprobe;          /* probes for kind 0 */
  gp_theta theta;
  const float* X;          /* host n x d */
  const float* y;          /* host n */
  const float* Xstar;      /* host m x d (kind 1) */
  int64_t m;
  int32_t cg_maxit;        /* CG iteration budget */
  int32_t nlanczos;
  double cg_rtol;
  uint64_t seed;
  int32_t prec;            /* arithmetic of the CG products (gp_precision) */
  int32_t slq_prec;        /* arithmetic of the SLQ products (gp_solve_opts.slq_prec) */
} gp_request;

typedef struct {
  gp_status status;
  int32_t cg_iters;
  double loss;
  double grad[3];
  double relres;
  double t_submit_s;       /* server clock (seconds) at submit */
  double t_start_s;        /* admitted to the device */
  double t_done_s;         /* result ready */
  float* mu;               /* caller's host buffer of m floats (kind 1), set before poll */
} gp_result;

/* Create a server on the current device with a device-memory budget and a
 * maximum number of concurrently resident requests (1..256; budget >= 1 MiB).
 * GP_ERR_OOM if the device pool cannot be reserved; GP_ERR_CUDA if a worker
 * cannot create its CUDA streams (every worker has reported before this call
 * returns, and on failure nothing is left running).  The server clock of
 * gp_result starts when this call returns. */
gp_status gp_server_create(size_t hbm_budget_bytes, int32_t max_slots, gp_server** out);
/* gp_server_create with batching: a worker that admits a loss + gradient
 * request with FP32 products also takes up to max_batch - 1 queued requests
 * that can share its grouped launches (same kernel, dimension class, nprobe
 * and nlanczos; work within a factor 16; blocks that fit the pool, least
 * work first) and runs them together as one gp_loss_and_grad_batch: one
 * grouped product launch per CG iteration, Lanczos step and gradient pass
 * for all of them.  Requests that arrive meanwhile queue for the next free
 * worker, as without batching.  Each result is the same as the request's
 * own gp_loss_and_grad (bit for bit when its padded width is one of the
 * grouped widths, e.g. 1 + nprobe = 17).  1 <= max_batch <= 64. */
gp_status gp_server_create_batched(size_t hbm_budget_bytes, int32_t max_slots, int32_t max_batch,
                                   gp_server** out);
/* Queue a request (host arrays copied at submit); returns a ticket.
 * GP_ERR_OOM if the request can never fit the budget. */
gp_status gp_server_submit(gp_server* srv, const gp_request* req, uint64_t* ticket);
/* Non-blocking: GP_OK and *res filled if the ticket is done (res->mu, if non-NULL,
 * receives the prediction), GP_ERR_TIMEOUT if still pending. */
gp_status gp_server_poll(gp_server* srv, uint64_t ticket, gp_result* res);
/* Block until every submitted request is done (GP_OK) or timeout_s elapses
 * (GP_ERR_TIMEOUT). */
gp_status gp_server_drain(gp_server* srv, double timeout_s);
/* Counters since creation. */
gp_status gp_server_get_stats(gp_server* srv, gp_server_stats* out);
/* Footprint in bytes the server charges a request (0 on invalid arguments). */
size_t gp_server_footprint(const gp_request* req);
/* Stop the workers after the running requests finish; queued requests are
 * dropped.  Frees the device pool and the pinned staging pool. */
gp_status gp_server_destroy(gp_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* GP_H */
