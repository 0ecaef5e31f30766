// FP32-pair instantiation of the residual kernel (residual.cuh), in its own
// unit so that it compiles in parallel with the FP64 one.
#include "residual.cuh"

namespace gp {

cudaError_t launch_residual_pair(const ResPlan& p, const ResArgs& a, cudaStream_t st) {
  return launch_residual_arith<kResPair>(p, a, st);
}

}  // namespace gp
