// Residual rows of an FP64 solution: planning, the fixed-order combine of the
// j-splits, and the FP64 instantiation of residual_kernel (residual.cuh).
#include <algorithm>

#include "residual.cuh"

namespace gp {

int num_sms();

namespace {

__global__ void residual_combine_kernel(const double* part, int split, int64_t m, int64_t m_pad,
                                        int w_part, const int64_t* rows, int64_t n, const float* B,
                                        int64_t ldb, const double* x64, int64_t ldx, int w,
                                        double f2, double snoise, double* R, int ldr, float* Bg) {
  const int64_t total = m_pad * ldr;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t k = e / ldr;
    const int c = static_cast<int>(e - k * ldr);
    double r = 0.0;
    float b = 0.0f;
    if (k < m && c < w) {
      const int64_t row = rows != nullptr ? rows[k] : k;
      if (row >= 0 && row < n) {
        double acc = 0.0;
        for (int s = 0; s < split; ++s) acc += part[(static_cast<int64_t>(s) * m_pad + k) * w_part + c];
        b = B[row * ldb + c];
        r = static_cast<double>(b) - (f2 * acc + snoise * x64[row * ldx + c]);
      } else {
        r = __longlong_as_double(0x7ff8000000000000ll);   // NaN for an invalid row index
      }
    }
    R[e] = r;
    if (Bg != nullptr) Bg[e] = b;
  }
}

int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int target_blocks() { return 4 * num_sms(); }

}  // namespace

ResPlan plan_residual(int64_t m, int64_t n, int w) {
  ResPlan p;
  p.cw = w == 1 ? 1 : (w <= 4 ? 4 : 8);
  p.col_groups = (w + p.cw - 1) / p.cw;
  p.w_part = p.col_groups * p.cw;
  p.m_pad = round_up64(m, kResRows);
  p.row_blocks = static_cast<int>(p.m_pad / kResRows);
  p.jtiles = (n + kResTile - 1) / kResTile;
  const int64_t units = static_cast<int64_t>(p.row_blocks) * p.col_groups;
  int64_t split = (target_blocks() + units - 1) / units;
  split = std::max<int64_t>(1, std::min<int64_t>(split, std::min<int64_t>(64, p.jtiles)));
  p.jt_per_split = (p.jtiles + split - 1) / split;
  p.split = static_cast<int>((p.jtiles + p.jt_per_split - 1) / p.jt_per_split);
  return p;
}

size_t residual_part_bytes_bound(int64_t n, int w) {
  const ResPlan p = plan_residual(n, n, w);
  // split * m_pad <= (target / units + 1) * m_pad <= target * kResRows + m_pad.
  const size_t rows = static_cast<size_t>(target_blocks()) * kResRows + static_cast<size_t>(p.m_pad);
  return rows * p.w_part * sizeof(double);
}

cudaError_t launch_residual(const ResPlan& p, ResArgs a, const ResidualCall& c, cudaStream_t st) {
  a.m_pad = p.m_pad;
  a.w_part = p.w_part;
  a.jtiles = p.jtiles;
  a.jt_per_split = p.jt_per_split;
  const cudaError_t e = c.arith == kResPair ? launch_residual_pair(p, a, st)
                                            : launch_residual_f64(p, a, st);
  if (e != cudaSuccess) return e;
  const int64_t total = p.m_pad * c.ldr;
  const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4096));
  residual_combine_kernel<<<blocks, 256, 0, st>>>(a.part, p.split, a.m, p.m_pad, p.w_part, a.rows,
                                                  a.n, c.B, c.ldb, a.x64, a.ldx, a.w, c.f2,
                                                  c.snoise, c.R, c.ldr, c.Bg);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_residual_f64(const ResPlan& p, const ResArgs& a, cudaStream_t st) {
  return launch_residual_arith<kResF64>(p, a, st);
}

}  // namespace gp
