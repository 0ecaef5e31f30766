// Tensor-core (tcgen05) form of the on-the-fly product.
#include "kmv_tc.cuh"

namespace gp {

SimtPlan plan_tc(int64_t nr, int64_t nc, int d, int w, int kernel, int) {
  return plan_simt(nr, nc, d, w, false, kernel);
}

cudaError_t launch_tc(const SimtPlan&, int, bool, int, const TcArgs&, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace gp
