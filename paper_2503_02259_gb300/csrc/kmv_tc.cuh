// Tensor-core (tcgen05) form of the on-the-fly product: declarations.
#pragma once

#include "gp_internal.cuh"

namespace gp {

struct TcArgs {
  const float* xr;
  const float* xc;
  const float* v;
  float* part_k;
  float* part_d;
  const int* active;
  int* err;
};

// Plan of the tensor-core product (fills the SimtPlan fields the epilogue and
// the workspace use: dp, w_pad, nr_pad, nc_pad, split).
SimtPlan plan_tc(int64_t nr, int64_t nc, int d, int w, int kernel, int prec);

// Returns cudaErrorNotSupported when the shape has no tensor-core form.
cudaError_t launch_tc(const SimtPlan& p, int kernel, bool grad, int prec, const TcArgs& a,
                      cudaStream_t st);

}  // namespace gp
