// Tensor-core (tcgen05) product: launch planning and dispatch over operand modes.
#include <algorithm>

#include "kmv_tc_kernel.cuh"

namespace gp {

cudaError_t launch_tc_mode1(const SimtPlan&, int, bool, const TcArgs&, cudaStream_t);
cudaError_t launch_tc_mode2(const SimtPlan&, int, bool, const TcArgs&, cudaStream_t);
cudaError_t launch_tc_mode3(const SimtPlan&, int, bool, const TcArgs&, cudaStream_t);
cudaError_t launch_tc_mode4(const SimtPlan&, int, bool, const TcArgs&, cudaStream_t);
int num_sms();

int tc_mode_for(int prec) {
  switch (prec) {
    case GP_PREC_TF32: return kTcTF32;
    case GP_PREC_BF16: return kTcBF16;
    case GP_PREC_TF32X3: return kTcTF32x3;
    case GP_PREC_BF16X3: return kTcBF16x3;
    default: return 0;
  }
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

SimtPlan plan_tc(int64_t nr, int64_t nc, int d, int w, int, int prec) {
  SimtPlan p{};
  p.dt = dim_template(d);
  p.dp = dim_padded(p.dt);
  p.tw = 0;
  p.ng = 0;
  p.w_pad = static_cast<int>(round_up(w, 16));
  p.bm = kTcM;
  p.nr_pad = round_up(nr, kPad);
  p.nc_pad = round_up(nc, kPad);
  p.row_tiles = static_cast<int>(p.nr_pad / kTcM);
  p.jtiles = static_cast<int>(p.nc_pad / tc_tile_cols(tc_mode_for(prec)));
  // Same balance rule as the SIMT plan: spread CTAs evenly over the SMs.
  const int nsm = num_sms();
  int best_s = 1;
  double best = 1e300;
  const int smax = std::min(p.jtiles, kMaxSplit);
  for (int s = 1; s <= smax; ++s) {
    const int jps = (p.jtiles + s - 1) / s;
    if ((p.jtiles + jps - 1) / jps != s) continue;
    const int64_t units = static_cast<int64_t>(p.row_tiles) * s;
    const double per_sm = static_cast<double>((units + nsm - 1) / nsm);
    const double cost = per_sm * (jps + 2.0) * (1.0 + 0.002 * s);
    if (cost < best) {
      best = cost;
      best_s = s;
    }
  }
  p.jt_per_split = (p.jtiles + best_s - 1) / best_s;
  p.split = (p.jtiles + p.jt_per_split - 1) / p.jt_per_split;
  return p;
}

size_t tc_vt_bytes(const SimtPlan& p, int prec) {
  switch (tc_mode_for(prec)) {
    // bytes per element x split parts of the B operand
    case kTcTF32: return static_cast<size_t>(p.nc_pad) * p.w_pad * 4;
    case kTcBF16: return static_cast<size_t>(p.nc_pad) * p.w_pad * 2 * 2;
    case kTcTF32x3: return static_cast<size_t>(p.nc_pad) * p.w_pad * 4 * 2;
    case kTcBF16x3: return static_cast<size_t>(p.nc_pad) * p.w_pad * 2 * 2;
    default: return 0;
  }
}

cudaError_t launch_tc(const SimtPlan& p, int kernel, bool grad, int prec, const TcArgs& a,
                      cudaStream_t st) {
  switch (tc_mode_for(prec)) {
    case kTcTF32: return launch_tc_mode1(p, kernel, grad, a, st);
    case kTcBF16: return launch_tc_mode2(p, kernel, grad, a, st);
    case kTcTF32x3: return launch_tc_mode3(p, kernel, grad, a, st);
    case kTcBF16x3: return launch_tc_mode4(p, kernel, grad, a, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace gp
