// Residual rows of a solution: R[k][c] = B[row_k][c] - (Kh X)[row_k][c],
// Kh = f^2 K + s I, for X held in FP64 (the outer residual of mixed-precision
// iterative refinement, and its checker).
//
// The O(n^2 w) part, sum_j K(x_row, x_j) X[j][c], runs in one of two
// arithmetics:
//  - kResF64: FP64 kernel entries (CUDA's double exp / sqrt) and FP64 sums.
//    GB300's FP64 pipe is slow, so this is the checker, not the solver path.
//  - kResPair: FP32-pair ("double-float") arithmetic of pair_arith.cuh: the
//    squared distance from the exact differences of the FP32 points, the
//    kernel entry by the table-driven pair exponential, the products K X[j] as
//    pairs, and compensated sums (two-sum accumulators per 64-point tile,
//    renormalised every four entries, added into a running pair sum), about
//    1e-14 relative per entry on the FP32 pipe.  Two column points are taken
//    per step in packed FP32x2 arithmetic (pair_arith2.cuh: each lane rounds
//    exactly as the scalar form), with one accumulator per lane, the two
//    lanes added at the end of each tile.
// Every block takes 128 rows k (one thread each), CW columns and one j range
// (split s); partial sums go to part[s][k][c] as FP64 values (a pair converts
// exactly) and a combine kernel sums the splits in a fixed order.
#pragma once

#include "gp_internal.cuh"
#include "pair_arith.cuh"
#include "pair_arith2.cuh"

namespace gp {

constexpr int kResF64 = 0;
constexpr int kResPair = 1;
constexpr int kResRows = 128;   // rows (threads) per block
constexpr int kResTile = 64;    // points j per shared-memory tile

struct ResArgs {
  const float* X;       // points, row-major n x d FP32 (unscaled)
  int64_t n;
  int d;
  int kernel;
  const int64_t* rows;  // row indices (NULL: row k = k)
  int64_t m;            // rows evaluated
  int64_t m_pad;        // rows rounded up to kResRows
  const double* x64;    // solution, n rows, leading dimension ldx, FP64
  int64_t ldx;
  int w;                // live columns
  int w_part;           // columns of a partial plane (column groups x CW)
  double* part;         // [split][m_pad][w_part]
  int64_t jtiles;       // tiles of kResTile points
  int64_t jt_per_split;
  double kc64;          // FP64 kernel constant: 1/(2 l^2) or sqrt(3)/l
  pa::fpair kc;         // the same as a pair
  int* err;             // set to 1 if a row index is out of range
};

template <int ARITH, int CW, int DMAX>
__global__ void __launch_bounds__(kResRows) residual_kernel(ResArgs a, pa::ExpConsts C) {
  __shared__ float sx[kResTile * DMAX];
  __shared__ __align__(16) unsigned char sv_raw[kResTile * CW * 8];
  __shared__ pa::ExpConsts sC;
  const int tid = threadIdx.x;
  if constexpr (ARITH == kResPair) {
    for (int e = tid; e < 64; e += blockDim.x) {
      sC.hi[e] = C.hi[e];
      sC.lo[e] = C.lo[e];
    }
    if (tid == 0) {
      sC.inv_ln2_64 = C.inv_ln2_64;
      sC.c0 = C.c0;
      sC.c1 = C.c1;
      sC.c2 = C.c2;
    }
  }
  const int64_t k = static_cast<int64_t>(blockIdx.x) * kResRows + tid;
  const int c0 = blockIdx.y * CW;
  const int s = blockIdx.z;
  const int64_t jt0 = s * a.jt_per_split;
  const int64_t jt1 = min(jt0 + a.jt_per_split, a.jtiles);
  const int d = a.d;

  int64_t row = -1;
  if (k < a.m) {
    row = a.rows != nullptr ? a.rows[k] : k;
    if (row < 0 || row >= a.n) {
      atomicExch(a.err, 1);
      row = -1;
    }
  }
  float xi[DMAX];
#pragma unroll
  for (int t = 0; t < DMAX; ++t) xi[t] = (row >= 0 && t < d) ? a.X[row * d + t] : 0.0f;

  double acc64[CW];
  pa::fpair run[CW], tacc[CW];
#pragma unroll
  for (int cc = 0; cc < CW; ++cc) {
    acc64[cc] = 0.0;
    run[cc] = {0.0f, 0.0f};
    tacc[cc] = {0.0f, 0.0f};
  }

  for (int64_t jt = jt0; jt < jt1; ++jt) {
    const int64_t j0 = jt * kResTile;
    __syncthreads();
    for (int e = tid; e < kResTile * DMAX; e += blockDim.x) {
      const int jj = e / DMAX, t = e - (e / DMAX) * DMAX;
      const int64_t j = j0 + jj;
      sx[e] = (j < a.n && t < d) ? a.X[j * d + t] : 0.0f;
    }
    for (int e = tid; e < kResTile * CW; e += blockDim.x) {
      const int jj = e / CW, cc = e - (e / CW) * CW;
      const int64_t j = j0 + jj;
      const int c = c0 + cc;
      const double v = (j < a.n && c < a.w) ? a.x64[j * a.ldx + c] : 0.0;
      if constexpr (ARITH == kResF64) {
        reinterpret_cast<double*>(sv_raw)[e] = v;
      } else {
        const pa::fpair p = pa::from_double(v);
        reinterpret_cast<float2*>(sv_raw)[e] = make_float2(p.hi, p.lo);
      }
    }
    __syncthreads();
    // Padded points (j >= n) meet zero solution values and add exact zeros.
    if constexpr (ARITH == kResF64) {
      const double* sv = reinterpret_cast<const double*>(sv_raw);
      for (int jj = 0; jj < kResTile; ++jj) {
        double r2 = 0.0;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
          if (t < d) {
            const double df = static_cast<double>(xi[t]) - static_cast<double>(sx[jj * DMAX + t]);
            r2 = fma(df, df, r2);
          }
        }
        double kv;
        if (a.kernel == GP_KERNEL_GAUSSIAN) {
          kv = exp(-r2 * a.kc64);
        } else {
          const double av = sqrt(r2) * a.kc64;
          kv = (1.0 + av) * exp(-av);
        }
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) acc64[cc] = fma(kv, sv[jj * CW + cc], acc64[cc]);
      }
    } else {
      const float2* sv = reinterpret_cast<const float2*>(sv_raw);
      pa2::fp2 tacc2[CW];
#pragma unroll
      for (int cc = 0; cc < CW; ++cc) tacc2[cc] = {pa2::bc(0.0f), pa2::bc(0.0f)};
      for (int jj = 0; jj < kResTile; jj += 4) {
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          // Entries jj + u (lane 0) and jj + u + 1 (lane 1).
          const pa2::fp2 r2 =
              pa2::sqdist<DMAX>(xi, sx + (jj + u) * DMAX, sx + (jj + u + 1) * DMAX, d);
          const pa2::fp2 kv = pa2::kernel_entry(r2, a.kernel, a.kc, sC);
#pragma unroll
          for (int cc = 0; cc < CW; ++cc) {
            const float2 xa = sv[(jj + u) * CW + cc], xb = sv[(jj + u + 1) * CW + cc];
            const pa2::fp2 p = pa2::mul(kv, pa2::fp2{make_float2(xa.x, xb.x), make_float2(xa.y, xb.y)});
            const pa2::fp2 t2 = pa2::two_sum(tacc2[cc].hi, p.hi);
            tacc2[cc] = {t2.hi, pa2::add(tacc2[cc].lo, pa2::add(t2.lo, p.lo))};
          }
        }
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) tacc2[cc] = pa2::two_sum(tacc2[cc].hi, tacc2[cc].lo);
      }
#pragma unroll
      for (int cc = 0; cc < CW; ++cc)
        run[cc] = pa::add(run[cc], pa::add(pa2::lane(tacc2[cc], 0), pa2::lane(tacc2[cc], 1)));
    }
  }
  if (k < a.m_pad) {
    double* out = a.part + (static_cast<int64_t>(s) * a.m_pad + k) * a.w_part + c0;
#pragma unroll
    for (int cc = 0; cc < CW; ++cc) {
      double v;
      if constexpr (ARITH == kResF64)
        v = acc64[cc];
      else
        v = pa::to_double(run[cc]);
      out[cc] = row >= 0 ? v : 0.0;
    }
  }
}

// Plan of one residual launch.
struct ResPlan {
  int cw;            // columns per thread: 1, 4 or 8
  int col_groups;
  int w_part;        // col_groups * cw
  int64_t m_pad;
  int row_blocks;
  int64_t jtiles;
  int split;
  int64_t jt_per_split;
};
ResPlan plan_residual(int64_t m, int64_t n, int w);
// Largest partial-plane bytes of any plan with m <= n rows.
size_t residual_part_bytes_bound(int64_t n, int w);

// Launch the product part: a.part = sum_j K x64 per split (sets the plan
// fields of a), then the combine: R[k][c] = B[row][c] - (f2 sum_s part + snoise
// x64[row][c]) for k < m, c < w, and 0 elsewhere in [m_pad][ldr]; Bg (if not
// NULL) receives B[row][c] in the same layout.
struct ResidualCall {
  int arith;
  const float* B;
  int64_t ldb;
  double f2, snoise;
  double* R;
  int ldr;
  float* Bg;
};
cudaError_t launch_residual(const ResPlan& p, ResArgs a, const ResidualCall& c, cudaStream_t st);

// Instantiation units (residual.cu: FP64, residual_pair.cu: pair).
cudaError_t launch_residual_f64(const ResPlan& p, const ResArgs& a, cudaStream_t st);
cudaError_t launch_residual_pair(const ResPlan& p, const ResArgs& a, cudaStream_t st);

template <int ARITH>
cudaError_t launch_residual_arith(const ResPlan& p, const ResArgs& a, cudaStream_t st) {
  static pa::ExpConsts consts = [] {
    pa::ExpConsts c;
    pa::make_exp_consts(c);
    return c;
  }();
  const dim3 grid(static_cast<unsigned>(p.row_blocks), static_cast<unsigned>(p.col_groups),
                  static_cast<unsigned>(p.split));
  const bool small_d = a.d <= 4;
#define GP_RES_L(CW, DM) residual_kernel<ARITH, CW, DM><<<grid, kResRows, 0, st>>>(a, consts)
  switch (p.cw) {
    case 1:
      if (small_d) GP_RES_L(1, 4); else GP_RES_L(1, 16);
      break;
    case 4:
      if (small_d) GP_RES_L(4, 4); else GP_RES_L(4, 16);
      break;
    default:
      if (small_d) GP_RES_L(8, 4); else GP_RES_L(8, 16);
      break;
  }
#undef GP_RES_L
  count_launch();
  return cudaGetLastError();
}

}  // namespace gp
