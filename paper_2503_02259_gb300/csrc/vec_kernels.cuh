// Declarations of the O(n w) kernels around the product: staging, epilogues,
// block-CG vector updates and reductions, probe generation, Lanczos/SLQ and the
// loss/gradient assembly.
#pragma once

#include "gp_internal.cuh"

namespace gp {

// Block-CG scalar state, resident in the workspace (one per solve).
constexpr int kMaxW = GP_MAX_COLS;
constexpr int kMaxK = GP_MAX_LANCZOS;

struct CgState {
  int n_active;          // columns still iterating
  int err;               // DevErr
  unsigned ticket;       // last-block counter of the current reduction
  int iter;              // iterations issued
  int maxit;
  int w;                 // live columns
  double rtol;
  int active[kMaxW];
  int iters[kMaxW];
  double rr[kMaxW];      // r^T r of the current residual
  double bn2[kMaxW];     // ||b||^2
  double alpha[kMaxW];
  double beta[kMaxW];
  double relres[kMaxW];
  double ahist[kMaxK][kMaxW];   // CG: alpha_j; Lanczos: diagonal alpha_j
  double bhist[kMaxK][kMaxW];   // CG: beta_j;  Lanczos: off-diagonal beta_j
  double h[kMaxK + 1][kMaxW];   // Lanczos: reorthogonalisation coefficients
  double tnorm[kMaxW];          // Lanczos: running estimate of ||T||
  // SLQ / gradient outputs
  double slq_val[kMaxW];     // per-probe SLQ values
  double dots[3][kMaxW];     // per-column W^T (dKh/dtheta V)
  double yalpha;
  double out[16];            // assembled results (see assemble kernel)
  unsigned ticket2;
  // Per-dimension length-scales: (s, f, l_1..l_d) quadratic terms, traces, gradient.
  double ard_quad[2 + GP_MAX_DIM];
  double ard_trace[2 + GP_MAX_DIM];
  double ard_grad[2 + GP_MAX_DIM];
  // Eq. 1 / Eq. 2 terms of a preconditioner in closed form (zero for M = I):
  double logdet_m;           // log|M|
  double trm[3];             // tr(M^-1 dM/dtheta), theta = s, f, l
  double vv[kMaxW];          // per-column v^T v of the preconditioned Hutchinson terms
  int group_counter;         // work counter of a grouped product (batched solves)
  unsigned bar_count;        // grid barrier of the fused CG step: arrivals
  unsigned bar_gen;          // grid barrier of the fused CG step: generation
};

// Reduction geometry for the O(n w) kernels.
constexpr int kRedThreads = 256;
constexpr int kLzDotBlocks = 128;
int red_blocks(int64_t n_pad);
// Doubles of reduction scratch needed by every kernel below for this shape.
size_t red_doubles(int64_t n_pad, int w_pad);

// Launchers (all asynchronous on `st`).
// Staged points: (X[i][t] - ref[t]) * cs[t] (cs: host array of d per-dimension scales).
cudaError_t launch_stage_points(const float* X, int64_t n, int d, int64_t ld, const float* ref,
                                const float* cs, int dp, int64_t n_pad, float* out, cudaStream_t st);
cudaError_t launch_pad_block(const float* V, int64_t n, int w, int64_t ldv, float* out,
                             int64_t n_pad, int w_pad, int col_off, cudaStream_t st);
cudaError_t launch_unpad_block(const float* in, int64_t n, int w, int w_pad, float* out,
                               int64_t ldo, int col_off, cudaStream_t st);
cudaError_t launch_probes(int64_t n, int p, uint64_t seed, float* Z, int64_t ldz, int col_off,
                          int64_t n_rows_fill, cudaStream_t st);

// Epilogue of a product: Y = cK * sum_s partK + cV * V;  dYf = cF * sum_s partK;
// dYl = cL * sum_s partD.  Outputs with a NULL pointer are skipped.  If *err != 0
// the outputs are filled with NaN (an asynchronous error report).
struct EpiArgs {
  const float* part_k;
  const float* part_d;
  int split;
  int64_t nr_pad;
  int w_pad;
  const float* v;        // padded V for the cV term (may be NULL if cV == 0)
  int64_t n;             // live rows
  int w;                 // live columns
  double cK, cV, cF, cL;
  float* y;  int64_t ldy;
  float* dyf; int64_t ldf;
  float* dyl; int64_t ldl;
  const int* err;
};
cudaError_t launch_epilogue(const EpiArgs& a, cudaStream_t st);

// Block CG (per-column CG with FP64 scalars) on padded [n_pad][w_pad] arrays.
cudaError_t launch_cg_init(CgState* S, const float* B, float* X, float* R, float* P, int64_t n_pad,
                           int w_pad, int w, int maxit, double rtol, double* red, cudaStream_t st);
// Q = f^2 sum partK + s P; pAp partials; alpha.
cudaError_t launch_cg_epi_alpha(CgState* S, const float* part_k, int split, const float* P,
                                float* Q, int64_t n_pad, int64_t n, int w_pad, double f2,
                                double snoise, double* red, cudaStream_t st);
// X += alpha P; R -= alpha Q; beta, convergence.
cudaError_t launch_cg_update(CgState* S, float* X, float* R, const float* P, const float* Q,
                             int64_t n_pad, int w_pad, double* red, cudaStream_t st);
// P = R + beta P.
cudaError_t launch_cg_pupdate(CgState* S, const float* R, float* P, int64_t n_pad, int w_pad,
                              cudaStream_t st);
// The three calls above as one cooperative launch with two grid barriers (the
// same arithmetic and summation order, so the same bits).  Usable when
// cg_step_fits(n_pad): every block of the reduction grid can be resident at once.
bool cg_step_fits(int64_t n_pad);
cudaError_t launch_cg_step(CgState* S, const float* part_k, int split, float* X, float* R, float* P,
                           float* Q, int64_t n_pad, int64_t n, int w_pad, double f2, double snoise,
                           double* red, cudaStream_t st);
// Preconditioned CG: X += alpha P; R -= alpha Q; relres from ||R|| (no beta).
cudaError_t launch_pcg_update(CgState* S, float* X, float* R, const float* P, const float* Q,
                              int64_t n_pad, int w_pad, double* red, cudaStream_t st);
// Preconditioned CG: rz = R^T Z per column, beta = rz / rz_prev (0 if first), S->rr = rz.
// Then launch_cg_pupdate with Z in place of R gives P = Z + beta P.
cudaError_t launch_pcg_rz(CgState* S, const float* R, const float* Z, int64_t n_pad, int w_pad,
                          bool first, double* red, cudaStream_t st);

// Lanczos with full reorthogonalisation, one independent process per column of
// a padded [n_pad][w_pad] block (columns [col0, col0 + p) active).
// Q: (k+1) planes of [n_pad][w_pad]; plane j holds q_j.
cudaError_t launch_lz_init(CgState* S, const float* B, float* Q0, int64_t n_pad, int w_pad, int col0,
                           int p, double* red, cudaStream_t st);
// W = f^2 sum partK + s q_j (rows < n); alpha_j = q_j^T W.
cudaError_t launch_lz_epi_alpha(CgState* S, const float* part_k, int split, const float* Qj,
                                float* W, int64_t n_pad, int64_t n, int w_pad, double f2,
                                double snoise, int j, double* red, cudaStream_t st);
// W -= alpha_j q_j + beta_{j-1} q_{j-1}.
cudaError_t launch_lz_three_term(CgState* S, float* W, const float* Q, int64_t n_pad, int w_pad,
                                 int j, cudaStream_t st);
// One classical Gram-Schmidt pass against q_0..q_j: h = Q^T W; W -= Q h.
cudaError_t launch_lz_reorth(CgState* S, float* W, const float* Q, int64_t n_pad, int w_pad, int j,
                             double* red, cudaStream_t st);
// beta_j = ||W||; truncation; q_{j+1} = W / beta_j.
cudaError_t launch_lz_norm_next(CgState* S, const float* W, float* Q, int64_t n_pad, int w_pad,
                                int j, int k, double* red, cudaStream_t st);

// Lanczos on M^-1/2 Kh M^-1/2 carried in the variables q = M^-1/2 qh, with the
// M-images P = M Q kept beside the basis Q:
// init: bn2 = z^T M^-1 z (Z = the probe block, V = M^-1 Z), q_0 = V / sqrt(bn2),
// p_0 = Z / sqrt(bn2).
cudaError_t launch_lz_init_m(CgState* S, const float* Z, const float* V, float* Q0, float* P0,
                             int64_t n_pad, int w_pad, int col0, int p, double* red, cudaStream_t st);
// One reorthogonalisation pass in the M-inner product: h = P^T U, U -= Q h, MU -= P h.
cudaError_t launch_lz_reorth_m(CgState* S, float* U, float* MU, const float* Q, const float* P,
                               int64_t n_pad, int w_pad, int j, double* red, cudaStream_t st);
// beta_j = sqrt(U^T MU); q_{j+1} = U / beta_j, p_{j+1} = MU / beta_j.
cudaError_t launch_lz_mnorm_next(CgState* S, const float* U, const float* MU, float* Q, float* P,
                                 int64_t n_pad, int w_pad, int j, int k, double* red, cudaStream_t st);
// out[c] = A_c^T B_c for every column (FP64, fixed order).
cudaError_t launch_plane_dots(CgState* S, const float* A, const float* B, int64_t n_pad, int w_pad,
                              double* out, double* red, cudaStream_t st);
// Subtract v^T dM/dtheta v from the probe columns' dots (see vec_kernels.cu).
cudaError_t launch_precond_corr(CgState* S, const double* U, const double* U2, int r, int w_pad, int p,
                                double f, cudaStream_t st);
// S->out[0] += S->logdet_m.
cudaError_t launch_add_logdet_m(CgState* S, cudaStream_t st);

// SLQ from the Lanczos coefficients of columns [col0, col0 + p): per-probe
// values into S->slq_val and (mean, stderr) into S->out[0..1].
cudaError_t launch_slq(CgState* S, int col0, int p, int k, cudaStream_t st);

// Gradient epilogue: sums of the fused product with V = [alpha | Z] dotted with
// W = [alpha | U] per column -> S->dots (scaled: s, f, l).
cudaError_t launch_grad_dots(CgState* S, const float* part_k, const float* part_d, int split,
                             const float* V, const float* W, int64_t n_pad, int w_pad, int w,
                             double cF, double cL, double* red, cudaStream_t st);
// y^T alpha -> S->yalpha (column 0 of B and X).
cudaError_t launch_yalpha(CgState* S, const float* B, const float* X, int64_t n_pad, int w_pad,
                          double* red, cudaStream_t st);
// Final assembly of loss and gradient into S->out (see vec_kernels.cu).
cudaError_t launch_assemble(CgState* S, int64_t n, int p, cudaStream_t st);
// S->dots[0][c] = sum_i A[i][c] B[i][c] (FP64, fixed order) for c < w.
cudaError_t launch_coldots(CgState* S, const float* A, const float* B, int64_t n_pad, int w_pad,
                           int w, double* red, cudaStream_t st);
// Replace column 0 of V (padded) by column 0 of X.
cudaError_t launch_copy_col0(const float* X, float* V, int64_t n_pad, int w_pad, cudaStream_t st);

// Posterior variance: B = f^2 K(X, X*_block) as padded columns (unscaled FP32
// points, rows < n, columns < w, zero elsewhere), and var[c] = f2 - B_c^T U_c.
// inv_l: host array of the d per-dimension 1 / l_t.
cudaError_t launch_cross_cols(const float* X, int64_t n, int d, const float* Xs, int w, int kernel,
                              const double* inv_l, double f2, float* B, int64_t n_pad, int w_pad,
                              cudaStream_t st);
cudaError_t launch_pred_var(CgState* S, const float* B, const float* U, int64_t n_pad, int w_pad,
                            int w, double f2, float* var, double* red, cudaStream_t st);

// Iterative refinement (the residual r64 = B - Kh x64 is in residual.cuh).
// S->rr[c] = ||r64_c||^2, S->bn2[c] = ||B_c||^2, S->relres[c] = sqrt(rr/bn2); rf = r64 as FP32.
cudaError_t launch_refine_norms(CgState* S, const double* r64, const float* B, float* rf,
                                int64_t n_pad, int w_pad, int w, double* red, cudaStream_t st);
// b = a widened to FP64 (total elements).
cudaError_t launch_widen(const float* a, double* b, int64_t total, cudaStream_t st);
// x64 += X (FP32 correction) for columns c < w.
cudaError_t launch_refine_update(double* x64, const float* X, int64_t n_pad, int w_pad, int w,
                                 cudaStream_t st);
// Xsol (n x w, ld w) = x64 rounded to FP32.
cudaError_t launch_refine_out(const double* x64, float* Xsol, int64_t n, int w_pad, int w,
                              cudaStream_t st);

}  // namespace gp
