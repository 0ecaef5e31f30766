// Gradient contraction for per-dimension length-scales (grad_ard.cu).
#pragma once

#include "vec_kernels.cuh"

namespace gp {

// c_t of dKh/dl_t = f^2 c_t E dd_t per dimension (host-filled).
struct ArdScales {
  double v[GP_MAX_DIM];
};

struct GradArdPlan {
  int64_t row_blocks;    // blocks of 128 rows
  int64_t jtiles;        // tiles of 64 points
  int64_t jt_per_split;
  int64_t split;
  int nq;                // quantities per block: 2 (1 + dimension template)
  size_t part_doubles;   // partial sums: row_blocks x split x nq
};
GradArdPlan plan_grad_ard(int64_t n_pad, int d);

// Contracts the entries of K and dK/dl_t with Gq = alpha alpha^T and
// Gt = U Z^T / p (V = [alpha | Z], W = [alpha | U], padded [n_pad][w_pad]
// FP32, staged points xs) and assembles S->ard_quad / ard_trace / ard_grad for
// (s, f, l_1..l_d); S->dots[0][c] must hold W_c^T V_c.  w = 1 + p <= 48.
// cudaErrorNotSupported for wider blocks.
cudaError_t launch_grad_ard(const GradArdPlan& g, int kernel, int w, int p, int d, int dp,
                            const float* xs, const float* V, const float* W, int64_t n_pad,
                            int w_pad, double* part, CgState* S, double f, const ArdScales& c,
                            cudaStream_t st);

}  // namespace gp
