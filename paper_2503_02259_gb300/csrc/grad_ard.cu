// Gradient of the training loss with per-dimension length-scales (ARD).
//
// With Theta = (s, f, l_1..l_d), the gradient equation of §Gaussian Processes
// (Eq. 2 with M = I) needs, for each parameter theta,
//   quad_theta  = alpha^T (dKh/dtheta) alpha,
//   trace_theta ~ (1/p) sum_c u_c^T (dKh/dtheta) z_c,   u_c = Kh^-1 z_c,
// i.e. quad_theta = sum_ij (dKh/dtheta)_ij Gq_ij and trace_theta = sum_ij
// (dKh/dtheta)_ij Gt_ij with Gq_ij = alpha_i alpha_j and Gt_ij = (1/p) sum_c
// U_ic Z_jc.  Instead of d derivative products (d x w outputs per row), this
// kernel evaluates each entry once and contracts it with Gq and Gt directly:
//   dKh/df_ij    = 2 f K_ij,
//   dKh/dl_t,ij  = f^2 c_t E_ij dd_t,ij,
// where dd_t is the squared difference of coordinate t in the staged
// (per-dimension scaled) points, E = K (Gaussian) or exp(-a) (Matern-3/2) and
// c_t = 2 / (l_t log2 e) (Gaussian) or 1 / l_t (Matern-3/2).  Per entry: the
// distance, the kernel, w FMAs for Gt and 2 (d + 1) accumulations.
//
// One thread per row i (its alpha_i and U_i / p in registers), tiles of 64
// points j (staged coordinates and the rows of V = [alpha | Z]) in shared
// memory; tile sums are added into running sums (FP32), the block sums its
// threads in FP64 in a fixed order, and a one-block finish kernel sums the
// blocks in a fixed order.
#include <algorithm>

#include "grad_ard.cuh"
#include "vec_kernels.cuh"

namespace gp {

int num_sms();

namespace {

constexpr int kGaThreads = 128;
constexpr int kGaTile = 64;

template <int KIND, int TW, int DMAX>
__global__ void __launch_bounds__(kGaThreads)
    grad_ard_kernel(const float* xs, const float* V, const float* W, int64_t n_pad, int w_pad,
                    int p, int d, int dp, int64_t jtiles, int64_t jt_per_split, double* part) {
  constexpr int NQ = 2 * (1 + DMAX);
  __shared__ float sx[kGaTile * 16];
  __shared__ float sv[kGaTile * TW];
  __shared__ double red[kGaThreads];
  const int tid = threadIdx.x;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kGaThreads + tid;
  const int s = blockIdx.y;
  const int64_t jt0 = s * jt_per_split;
  const int64_t jt1 = min(jt0 + jt_per_split, jtiles);

  float xi[DMAX];
#pragma unroll
  for (int t = 0; t < DMAX; ++t) xi[t] = t < dp ? xs[pt_index(i, t, dp)] : 0.0f;
  // alpha_i and U_ic / p (column 0 of W is alpha, columns 1..p are U).
  float a[TW];
  const float inv_p = p > 0 ? 1.0f / static_cast<float>(p) : 0.0f;
#pragma unroll
  for (int c = 0; c < TW; ++c) {
    const float v = c < w_pad ? W[i * w_pad + c] : 0.0f;
    a[c] = c == 0 ? v : v * inv_p;
  }
  float run[NQ], acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) run[q] = acc[q] = 0.0f;

  for (int64_t jt = jt0; jt < jt1; ++jt) {
    const int64_t j0 = jt * kGaTile;
    __syncthreads();
    // The 64 points are two consecutive 32-point tiles of the staged layout.
    const float* src = xs + (j0 >> 5) * (32 * dp);
    for (int e = tid; e < kGaTile * dp; e += kGaThreads) sx[e] = src[e];
    for (int e = tid; e < kGaTile * TW; e += kGaThreads) {
      const int jj = e / TW, c = e - (e / TW) * TW;
      sv[e] = c < w_pad ? V[(j0 + jj) * w_pad + c] : 0.0f;
    }
    __syncthreads();
    for (int jj = 0; jj < kGaTile; ++jj) {
      const float* xj = sx + (jj >> 5) * (32 * dp) + (jj & 31);
      float dd[DMAX];
      float qd = 0.0f;
#pragma unroll
      for (int t = 0; t < DMAX; ++t) {
        dd[t] = 0.0f;
        if (t < d) {
          const float df = xi[t] - xj[t * 32];
          dd[t] = df * df;
          qd += dd[t];
        }
      }
      float K, E;
      if constexpr (KIND == GP_KERNEL_GAUSSIAN) {
        K = dev::ex2_approx(-qd);
        E = K;
      } else {
        const float av = dev::sqrt_approx(qd);
        E = dev::ex2_approx(av * -1.4426950408889634f);
        K = fmaf(av, E, E);
      }
      const float* vj = sv + jj * TW;
      const float gq = a[0] * vj[0];
      float gt = 0.0f;
#pragma unroll
      for (int c = 1; c < TW; ++c) gt = fmaf(a[c], vj[c], gt);
      acc[0] = fmaf(K, gq, acc[0]);
      acc[1] = fmaf(K, gt, acc[1]);
      const float hq = E * gq, ht = E * gt;
#pragma unroll
      for (int t = 0; t < DMAX; ++t) {
        acc[2 + 2 * t] = fmaf(hq, dd[t], acc[2 + 2 * t]);
        acc[3 + 2 * t] = fmaf(ht, dd[t], acc[3 + 2 * t]);
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      run[q] += acc[q];
      acc[q] = 0.0f;
    }
  }
  // Block sums in FP64 (fixed order), one partial per quantity and block.
  const int64_t blk = static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    red[tid] = static_cast<double>(run[q]);
    __syncthreads();
    for (int h = kGaThreads / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) part[blk * NQ + q] = red[0];
    __syncthreads();
  }
}

// Sums the blocks' partials in order and assembles quad, trace and the
// gradient of (s, f, l_1..l_d) into S->ard_*; the s terms come from
// S->dots[0] (alpha^T alpha and u_c^T z_c).
__global__ void grad_ard_finish_kernel(CgState* S, const double* part, int64_t nblocks, int nq,
                                       int p, int d, double f, ArdScales c) {
  __shared__ double tot[2 * (1 + GP_MAX_DIM)];
  const int q = threadIdx.x;
  if (q < nq) {
    double acc = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) acc += part[b * nq + q];
    tot[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tr_s = 0.0;
  for (int cc = 1; cc <= p; ++cc) tr_s += S->dots[0][cc];
  tr_s = p > 0 ? tr_s / p : 0.0;
  S->ard_quad[0] = S->dots[0][0];
  S->ard_trace[0] = tr_s;
  S->ard_quad[1] = 2.0 * f * tot[0];
  S->ard_trace[1] = 2.0 * f * tot[1];
  for (int t = 0; t < d; ++t) {
    S->ard_quad[2 + t] = f * f * c.v[t] * tot[2 + 2 * t];
    S->ard_trace[2 + t] = f * f * c.v[t] * tot[3 + 2 * t];
  }
  for (int k = 0; k < 2 + d; ++k) S->ard_grad[k] = 0.5 * (-S->ard_quad[k] + S->ard_trace[k]);
}

template <int KIND, int TW>
cudaError_t launch_tw(int d, dim3 grid, const float* xs, const float* V, const float* W,
                      int64_t n_pad, int w_pad, int p, int dp, int64_t jtiles, int64_t jps,
                      double* part, cudaStream_t st) {
  if (d <= 4)
    grad_ard_kernel<KIND, TW, 4><<<grid, kGaThreads, 0, st>>>(xs, V, W, n_pad, w_pad, p, d, dp,
                                                               jtiles, jps, part);
  else
    grad_ard_kernel<KIND, TW, 16><<<grid, kGaThreads, 0, st>>>(xs, V, W, n_pad, w_pad, p, d, dp,
                                                                jtiles, jps, part);
  return cudaGetLastError();
}

}  // namespace

GradArdPlan plan_grad_ard(int64_t n_pad, int d) {
  GradArdPlan g;
  g.row_blocks = n_pad / kGaThreads;
  g.jtiles = n_pad / kGaTile;
  const int64_t target = 4 * static_cast<int64_t>(num_sms());
  int64_t split = (target + g.row_blocks - 1) / g.row_blocks;
  split = std::max<int64_t>(1, std::min<int64_t>(split, std::min<int64_t>(64, g.jtiles)));
  g.jt_per_split = (g.jtiles + split - 1) / split;
  g.split = (g.jtiles + g.jt_per_split - 1) / g.jt_per_split;
  g.nq = 2 * (1 + (d <= 4 ? 4 : 16));
  g.part_doubles = static_cast<size_t>(g.row_blocks) * g.split * g.nq;
  return g;
}

cudaError_t launch_grad_ard(const GradArdPlan& g, int kernel, int w, int p, int d, int dp,
                            const float* xs, const float* V, const float* W, int64_t n_pad,
                            int w_pad, double* part, CgState* S, double f, const ArdScales& c,
                            cudaStream_t st) {
  const dim3 grid(static_cast<unsigned>(g.row_blocks), static_cast<unsigned>(g.split));
  cudaError_t e;
  if (w > 48 || d > GP_MAX_DIM) return cudaErrorNotSupported;
  if (kernel == GP_KERNEL_GAUSSIAN)
    e = w <= 16 ? launch_tw<GP_KERNEL_GAUSSIAN, 16>(d, grid, xs, V, W, n_pad, w_pad, p, dp,
                                                     g.jtiles, g.jt_per_split, part, st)
                : launch_tw<GP_KERNEL_GAUSSIAN, 48>(d, grid, xs, V, W, n_pad, w_pad, p, dp,
                                                     g.jtiles, g.jt_per_split, part, st);
  else
    e = w <= 16 ? launch_tw<GP_KERNEL_MATERN32, 16>(d, grid, xs, V, W, n_pad, w_pad, p, dp,
                                                     g.jtiles, g.jt_per_split, part, st)
                : launch_tw<GP_KERNEL_MATERN32, 48>(d, grid, xs, V, W, n_pad, w_pad, p, dp,
                                                     g.jtiles, g.jt_per_split, part, st);
  count_launch();
  if (e != cudaSuccess) return e;
  grad_ard_finish_kernel<<<1, 64, 0, st>>>(S, part, static_cast<int64_t>(g.row_blocks) * g.split,
                                           g.nq, p, d, f, c);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gp
