// Tensor-core (tcgen05) form of the on-the-fly product: declarations.
#pragma once

#include "gp_internal.cuh"

namespace gp {

// Arithmetic of the tensor-core contraction.
enum TcMode : int {
  kTcTF32 = 1,    // TF32 operands, FP32 accumulation in tensor memory
  kTcBF16 = 2,    // BF16 operands, FP32 accumulation
  kTcTF32x3 = 3,  // hi/lo TF32 split (A_hi B_hi + A_hi B_lo + A_lo B_hi): FP32-level accuracy
  kTcBF16x3 = 4   // the same split with BF16 parts
};

// Library precision enum -> mode (GP_PREC_FP32 has no tensor-core mode).
int tc_mode_for(int prec);

struct TcArgs {
  const float* xr;   // row points, AoS [nr_pad][dp], scaled
  const float* xc;   // column points, AoS [nc_pad][dp], scaled
  const float* v;    // [nc_pad][w_pad] FP32 multivector
  void* vt;          // scratch: V re-laid out per j tile as the MMA B operand
  float* part_k;     // [S][nr_pad][w_pad]
  float* part_d;     // [S][nr_pad][w_pad] (grad only)
  const int* active; // optional early-exit flag (0 = skip)
  int* err;          // device status word
};

// Plan of the tensor-core product (fills the SimtPlan fields the epilogue and
// the workspace use: dt, dp, w_pad (= w rounded up to 16), nr_pad, nc_pad,
// row_tiles, jtiles (32-point tiles), split, jt_per_split).
SimtPlan plan_tc(int64_t nr, int64_t nc, int d, int w, int kernel, int prec);

// Bytes of the B-operand scratch (TcArgs::vt) for a plan.
size_t tc_vt_bytes(const SimtPlan& p, int prec);

// Stage V into the B-operand layout and run the product (two launches).
// Returns cudaErrorNotSupported when the shape has no tensor-core form.
cudaError_t launch_tc(const SimtPlan& p, int kernel, bool grad, int prec, const TcArgs& a,
                      cudaStream_t st);

}  // namespace gp
