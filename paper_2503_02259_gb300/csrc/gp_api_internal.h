// Host-side declarations shared by the C-ABI units (not installed).
#pragma once

#include "gp_internal.cuh"

namespace gp {

// Launch plan for a product of nr rows x nc columns x w: the SIMT tiling for FP32
// and the tensor-core tiling for TF32 / BF16.
SimtPlan plan_for(int64_t nr, int64_t nc, int d, int w, bool grad, int kernel, int prec);

}  // namespace gp

// Mixed-precision iterative refinement (refine.cu).
// Writes the solution to Xsol (FP32) and/or X64 (FP64); either may be NULL.
gp_status refine_solve(const gp_problem* prob, const float* B, int32_t w, float* Xsol, double* X64,
                       const gp_solve_opts* opts, int32_t* iters, double* relres, void* ws,
                       size_t ws_bytes, cudaStream_t st);
