// Nystrom preconditioner for the CG solves: M = s I + L L^T, where L (n x r)
// is the rank-r partial Cholesky factor of f^2 K with greedy diagonal pivoting
// (each step takes the point with the largest residual diagonal, so the
// pivots are landmark points spread over the data).  The paper's PCG
// (§Gaussian Processes) leaves M open and its own choice, AFN, also starts
// from a Nystrom factor on chosen landmarks; this is that factor alone, used
// for the solves.  M^-1 V = (V - L C^-1 L^T V) / s with C = s I + L^T L (the
// Woodbury identity); C^-1 is formed once in FP64.
//
// Arithmetic.  L is stored in FP32.  Every sum that the Woodbury form
// cancels (the dot products of the factor steps, the Gram matrix L^T L,
// L^T V and L T) is taken with exact FP32 products and FP32-pair sums, so
// the preconditioner applied is the exact inverse of s I + L L^T for the
// stored L up to the final rounding of M^-1 V to FP32: in the directions of
// L's large singular values sigma the result is s / (s + sigma^2) times the
// input, and a plain FP32 sum there would carry a relative error of about
// u sigma^2 / s (1e-1 at sigma^2 = 1.6e4, s = 1e-2).
#pragma once

#include "gp_internal.cuh"
#include "pair_arith.cuh"

namespace gp {

constexpr int kNysMaxRank = GP_MAX_PRECOND_RANK;

// Scalar state of the factorisation (device).
struct NysState {
  int rank;           // columns built
  int stop;           // the factor has stopped (tolerance or rank reached)
  int err;            // DevErr of the factor or of C's Cholesky factorisation
  int pad0;
  long long pivot;    // pivot of the next step
  double dp;          // its residual diagonal
  double ddp;         // d(dp)/dl (derivative factor only)
  unsigned ticket;    // last-block counter
  unsigned pad1;
  double logdet_c;    // log|C|
  double tr_w;        // tr(C^-1)
  double tr_wh;       // <C^-1, L^T dL/dl> (derivative factor only)
};

// Inputs of the factor: the problem's points and kernel.
struct NysProblem {
  const float* X;     // device, n x d row-major
  int64_t n;
  int d;
  int kernel;
  double f, l, s;
  const double* ls;   // host per-dimension length-scales (NULL: isotropic l)
};

// Workspace layout (all sizes for the largest rank kmax and width w_pad).
struct NysWs {
  float* xs;          // [n_pad][d] points, divided by l_t under per-dimension scales
  float* Lt;          // [kmax][n_pad]: column j of L is row j
  double* dg;         // [n_pad] residual diagonal
  float* prow;        // [kmax] row of L at the next pivot
  long long* piv;     // [kmax] pivots
  double* amax_v;     // [step blocks] block maxima of the residual diagonal
  long long* amax_i;  // [step blocks] their indices
  NysState* S;
  double* C;          // [kmax][kmax]: s I + L^T L, then its Cholesky factor (lower)
                      // with the transposed factor in the upper triangle
  double* cdiag;      // [kmax] sqrt of the pivots of C's factorisation
  double* Winv;       // [kmax][kmax]: C^-1
  double* gpart;      // Gram partial sums
  double* upart;      // [chunks][kmax][w_pad] partial sums of L^T V
  double* U;          // [kmax][w_pad] L^T V
  float* Tp;          // [kmax][w_pad][2] C^-1 L^T V as FP32 pairs
  double* tred;       // block partials of the <C^-1, L^T dL/dl> reduction
  // Derivative factor (loss and gradient with the preconditioner):
  float* Ldt;         // [kmax][n_pad]: column j of dL/dl is row j
  float* dprow;       // [kmax] row of dL/dl at the next pivot
  double* gpart2;     // partial sums of L^T dL/dl
  double* U2;         // [kmax][w_pad] (dL/dl)^T V
  int64_t n_pad;
  int kmax, w_pad, d;
  // Columns of the V / Z planes that the apply computes (a multiple of 4,
  // <= w_pad): a solve sets it to its own width, rounded up to 4, when the
  // planes are padded wider for a tensor-core product; the apply writes zeros
  // to the columns from w_live to w_pad.  carve_nys sets it to w_pad.
  int w_live;
  bool deriv;
  size_t bytes;
};

size_t nys_bytes(int64_t n_pad, int d, int kmax, int w_pad, bool deriv = false);
NysWs carve_nys(void* base, int64_t n_pad, int d, int kmax, int w_pad, bool deriv = false);

// Builds L (at most kmax columns; stops early when the largest residual
// diagonal is <= tol_abs), C = s I + L^T L, its FP64 Cholesky factor and C^-1.
// Synchronises `st`; *rank = columns built; returns cudaErrorInvalidValue with
// *dev_err != 0 if C's factorisation met a non-positive pivot.
cudaError_t nys_build(const NysWs& W, const NysProblem& P, int kmax, double tol_abs, int* rank,
                      int* dev_err, cudaStream_t st);
// With a workspace carved with deriv = true, nys_build also forms dL/dl (the
// forward derivative of every column step with the pivots held fixed:
// dL[:, j] = (dS_p - L[:, j] d(d_p)/2 / sqrt(d_p)) / sqrt(d_p), dS_p the derivative of
// the Schur column, isotropic length-scale only) and <C^-1, L^T dL/dl>; every
// build forms log|C| and tr(C^-1).

// Terms of Eq. 1 / Eq. 2 that the preconditioner gives in closed form (pivots
// fixed; M = s I + L L^T, C = s I + L^T L, r = rank):
//   log|M| = (n - r) log s + log|C|;
//   tr(M^-1 dM/ds) = (n - r)/s + tr(C^-1);  tr(M^-1 dM/df) = (2/f)(r - s tr(C^-1));
//   tr(M^-1 dM/dl) = 2 tr(C^-1 L^T dL/dl).
// Written on the device into logdet_m[0] and trm[0..2].
cudaError_t nys_closed_terms(const NysWs& W, int rank, int64_t n, double s, double f,
                             double* logdet_m, double* trm, cudaStream_t st);

// Probe block B[:, col0 .. col0 + p) = L e1 + sqrt(s) e2 ~ N(0, M) (rows >= n
// zero), e1 = rows [n, n + rank) and e2 = rows [0, n) of a standard normal
// block: `eps` (device, (n + kmax) x p row-major, ld p) when non-NULL, else
// generated: e[i][c] = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller) with u1, u2
// from the SplitMix64 hash of (seed ^ 2^39, c, 2i) and (seed ^ 2^39, c, 2i + 1).
// Uses the workspace's Tp; B is [n_pad][w_pad].
cudaError_t nys_probes(const NysWs& W, int rank, int64_t n, double s, const float* eps, uint64_t seed,
                       int p, float* B, int col0, cudaStream_t st);

// U = L^T V (or (dL/dl)^T V when `deriv_matrix`) for the [n_pad][w_pad] block
// V, into U [rank][w_pad] (FP64, exact products and pair sums).
cudaError_t nys_lt_times(const NysWs& W, int rank, bool deriv_matrix, const float* V, double* U,
                         cudaStream_t st);

// Z = M V = s V + L (L^T V) (exact products and pair sums), same conventions
// as nys_apply; V and Z may not alias.
cudaError_t nys_apply_m(const NysWs& W, int rank, int64_t n, double s, const float* V, float* Z,
                        const int* active, cudaStream_t st);

// Z = M^-1 V on padded [n_pad][w_pad] blocks (rows >= n of Z are zero).  If
// `active` is non-NULL and *active == 0 the kernels exit (converged solves).
cudaError_t nys_apply(const NysWs& W, int rank, int64_t n, double s, const float* V, float* Z,
                      const int* active, cudaStream_t st);

}  // namespace gp
