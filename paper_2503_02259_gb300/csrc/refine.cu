// Mixed-precision iterative refinement around the tensor-core CG.
#include "gp_api_internal.h"

gp_status refine_solve(const gp_problem*, const float*, int32_t, float*, const gp_solve_opts*,
                       int32_t*, double*, void*, size_t, cudaStream_t) {
  gp::set_error("iterative refinement is not built yet");
  return GP_ERR_UNIMPLEMENTED;
}
