// Nystrom preconditioner M = s I + L L^T (see nystrom.cuh): the partial
// pivoted Cholesky factor L of f^2 K, the Gram matrix C = s I + L^T L, C's FP64
// Cholesky factorisation and inverse, and the application M^-1 V by the
// Woodbury identity.
//
// Accurate dot products: acc_prod is the Dot2 scheme of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005): the
// exact product a b = p + e (TwoProd), TwoSum of p into the running high part,
// and the two rounding errors summed into the low part.  The result carries the
// error of a dot product computed in twice the working precision.
#include <math.h>

#include <algorithm>
#include <climits>

#include "nystrom.cuh"
#include "pair_arith2.cuh"

namespace gp {

namespace {

constexpr int kStepThreads = 256;
// Rows per thread of a factor step: 4 (one float4 per column of L), except
// for the derivative factor when four rows would leave fewer than about four
// blocks per SM: then 1 (more blocks and loads in flight for its two streams).
// Measured at n = 2e5, rank 1500: the derivative build is faster with 1 row
// (a preconditioned loss 2.88 -> 2.72 s), the plain factor slower (0.42 ->
// 0.52 s, four times the shared-memory reads of the pivot row), so the plain
// factor always takes 4.
constexpr int kStepRowsWide = 4;
constexpr int kStepWideMinBlocks = 152 * 4;
constexpr int kStepBatch = 8;                     // columns of L loaded ahead per thread
constexpr int kGT = 64;                           // Gram tile (columns of L)
constexpr int kGK = 32;                           // Gram rows per shared-memory slab
constexpr int kLtvChunk = 4096;                   // rows per block of L^T V (chunk bound of upart)
constexpr int kLtM = 64;                          // columns of L per block of L^T V
constexpr int kLtPairs = 20;                      // column pairs of V per block of L^T V (at most)
constexpr int kZPairs = 10;                       // column pairs of Z per thread (at most)
constexpr int kZTile = 128;                       // rows of T staged per pass of the Z kernel
constexpr int kInvWarps = 2;                      // columns of C^-1 per block
constexpr int kRedCap = 152 * 16;                 // blocks of a grid_for reduction

__device__ __forceinline__ void acc_prod(pa::fpair& acc, float a, float b) {
  const pa::fpair p = pa::two_prod(a, b);
  const pa::fpair s = pa::two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo = pa::add(acc.lo, pa::add(s.lo, p.lo));
}

// acc += a (thi + tlo): the product with the high part exact, the low part's
// product folded into the error term.
__device__ __forceinline__ void acc_prod_pair(pa::fpair& acc, float a, float thi, float tlo) {
  const pa::fpair p = pa::two_prod(a, thi);
  const pa::fpair s = pa::two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo = pa::add(acc.lo, pa::add(s.lo, pa::fma_(a, tlo, p.lo)));
}

__device__ __forceinline__ void renorm(pa::fpair& a) { a = pa::fast_two_sum(a.hi, a.lo); }

// acc_prod and acc_prod_pair on two columns at once in packed FP32x2
// arithmetic (pair_arith2.cuh): each lane performs the scalar form's rounded
// operations, so each column's sum is the scalar Dot2 sum bit for bit.
__device__ __forceinline__ void acc_prod2(pa2::fp2& acc, float a, float2 b) {
  const pa2::fp2 p = pa2::two_prod(pa2::bc(a), b);
  const pa2::fp2 s = pa2::two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo = pa2::add(acc.lo, pa2::add(s.lo, p.lo));
}

__device__ __forceinline__ void acc_prod_pair2(pa2::fp2& acc, float a, float2 thi, float2 tlo) {
  const pa2::f2 a2 = pa2::bc(a);
  const pa2::fp2 p = pa2::two_prod(a2, thi);
  const pa2::fp2 s = pa2::two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo = pa2::add(acc.lo, pa2::add(s.lo, pa2::fma_(a2, tlo, p.lo)));
}

__device__ __forceinline__ void renorm2(pa2::fp2& a) { a = pa2::fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ pa::fpair warp_sum_pair(pa::fpair v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const pa::fpair w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = pa::add(v, w);
  }
  return v;
}

// (v, i) <- the better of (v, i) and (v2, i2): larger value, then smaller index.
__device__ __forceinline__ void better(double& v, long long& i, double v2, long long i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

__device__ __forceinline__ void warp_argmax(double& v, long long& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
    better(v, i, v2, i2);
  }
}

// True in exactly one block: the last to arrive (its reads see every block's writes).
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x * gridDim.y * gridDim.z - 1);
    if (am_last) *ticket = 0u;
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

struct StageScales {
  float v[GP_MAX_DIM];
};

// ----------------------------------------------------------- factor steps --

// xs = scaled points; dg = f^2 (the diagonal of f^2 K, k(0) = 1); state reset
// with the first pivot 0 (every diagonal entry is equal, and ties go to the
// smallest index).
__global__ void nys_init_kernel(const float* X, int64_t n, int d, const StageScales sc,
                                int64_t n_pad, double f2, float* xs, double* dg, NysState* S) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_pad;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int t = 0; t < d; ++t) xs[i * d + t] = i < n ? X[i * d + t] * sc.v[t] : 0.0f;
    dg[i] = i < n ? f2 : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->rank = 0;
    S->stop = 0;
    S->err = 0;
    S->pivot = 0;
    S->dp = f2;
    S->ddp = 0.0;
    S->ticket = 0u;
  }
}

struct StepArgs {
  const float* xs;
  int64_t n, n_pad;
  int d, kernel;
  pa::fpair kc;       // kernel constant (kernel_pair_const)
  pa::fpair dlc;      // derivative constant: 1/l^3 (Gaussian) or 1/l (Matern-3/2)
  double f2, tol_abs;
  int kmax;
  float* Lt;
  double* dg;
  float* prow;
  long long* piv;
  double* amax_v;
  long long* amax_i;
  NysState* S;
  float* Ldt;         // derivative factor (DERIV only)
  float* dprow;
};

// k(r) and dk/dl from r^2 in pair arithmetic (isotropic l):
// Gaussian k = exp(-r^2 kc), dk/dl = k r^2 / l^3; Matern-3/2 with a = r kc:
// k = (1 + a) e^-a, dk/dl = a^2 e^-a / l.
__device__ __forceinline__ void kernel_and_dl(pa::fpair r2, int kernel, pa::fpair kc, pa::fpair dlc,
                                              const pa::ExpConsts& C, pa::fpair& k, pa::fpair& dk) {
  if (kernel == 0) {
    k = pa::exp(pa::neg(pa::mul(r2, kc)), C);
    dk = pa::mul(pa::mul(k, r2), dlc);
  } else {
    const pa::fpair a = pa::mul(pa::sqrt(r2), kc);
    const pa::fpair e = pa::exp(pa::neg(a), C);
    k = pa::mul(pa::add_f(a, 1.0f), e);
    dk = pa::mul(pa::mul(pa::mul(a, a), e), dlc);
  }
}

// Step j: with p the current pivot and d_p its residual diagonal,
//   L[i][j] = (f^2 k(x_i, x_p) - sum_{m<j} L[i][m] L[p][m]) / sqrt(d_p),
//   d_i -= L[i][j]^2 (d_p = 0), and the next pivot = argmax_i d_i.
// The kernel entry is the pair exponential of the compensated residual and
// the dot product is Dot2, so the column is exact for the stored (FP32)
// earlier columns up to its final rounding; d is kept in FP64 as the exact
// residual diagonal of the stored factor.  With DERIV the same step also
// forms column j of dL/dl (pivots fixed):
//   dS_i = f^2 dk/dl(x_i, x_p) - sum_{m<j} (dL[i][m] L[p][m] + L[i][m] dL[p][m]),
//   dL[i][j] = (dS_i - L[i][j] dd_p / 2 / sqrt(d_p)) / sqrt(d_p),
// with dd_p = -2 sum_m L[p][m] dL[p][m] (dk/dl = 0 at r = 0), formed by the
// previous step's last block.
template <int ROWS>
__device__ __forceinline__ void load_rows(const float* p, float (&out)[ROWS]) {
  if constexpr (ROWS == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    out[0] = t.x;
    out[1] = t.y;
    out[2] = t.z;
    out[3] = t.w;
  } else {
    out[0] = *p;
  }
}

template <int ROWS>
__device__ __forceinline__ void store_rows(float* p, const float (&v)[ROWS]) {
  if constexpr (ROWS == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *p = v[0];
}

template <int DMAX, bool DERIV, int ROWS>
__global__ void __launch_bounds__(kStepThreads)
    nys_step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ pa::ExpConsts C, int j) {
  extern __shared__ float sp[];   // row p of L, then (DERIV) row p of dL/dl; columns < j
  NysState* S = a.S;
  if (S->stop) return;
  const long long p = S->pivot;
  const double dp = S->dp;
  const double ddp = DERIV ? S->ddp : 0.0;
  float* sdp = sp + a.kmax;
  for (int m = threadIdx.x; m < j; m += blockDim.x) {
    sp[m] = a.prow[m];
    if constexpr (DERIV) sdp[m] = a.dprow[m];
  }
  float xp[DMAX];
#pragma unroll
  for (int t = 0; t < DMAX; ++t) xp[t] = t < a.d ? a.xs[p * a.d + t] : 0.0f;
  __syncthreads();
  const int64_t i0 = (static_cast<int64_t>(blockIdx.x) * kStepThreads + threadIdx.x) * ROWS;
  double best = -INFINITY;
  long long besti = LLONG_MAX;
  if (i0 < a.n_pad) {
    pa::fpair acc[ROWS] = {};
    pa::fpair dacc[ROWS] = {};
    const float* col = a.Lt + i0;
    const float* dcol = DERIV ? a.Ldt + i0 : nullptr;
    // Batches of columns: all loads of a batch are issued before the first
    // is used, so that enough bytes are in flight to stream L at the memory's
    // rate.
    constexpr int kB = (ROWS == 1 ? 2 * kStepBatch : kStepBatch) / (DERIV ? 2 : 1);
    int m = 0;
    for (; m + kB <= j; m += kB) {
      float l[kB][ROWS], dl[kB][ROWS];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        load_rows<ROWS>(col + static_cast<int64_t>(m + u) * a.n_pad, l[u]);
        if constexpr (DERIV) load_rows<ROWS>(dcol + static_cast<int64_t>(m + u) * a.n_pad, dl[u]);
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const float b = sp[m + u];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) acc_prod(acc[q], l[u][q], b);
        if constexpr (DERIV) {
          const float db = sdp[m + u];
#pragma unroll
          for (int q = 0; q < ROWS; ++q) {
            acc_prod(dacc[q], dl[u][q], b);
            acc_prod(dacc[q], l[u][q], db);
          }
        }
      }
    }
    for (; m < j; ++m) {
      float l[ROWS], dl[ROWS];
      load_rows<ROWS>(col + static_cast<int64_t>(m) * a.n_pad, l);
      const float b = sp[m];
#pragma unroll
      for (int q = 0; q < ROWS; ++q) acc_prod(acc[q], l[q], b);
      if constexpr (DERIV) {
        load_rows<ROWS>(dcol + static_cast<int64_t>(m) * a.n_pad, dl);
        const float db = sdp[m];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
          acc_prod(dacc[q], dl[q], b);
          acc_prod(dacc[q], l[q], db);
        }
      }
    }
    const double inv = 1.0 / sqrt(dp);
    float out[ROWS], dout[ROWS];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int64_t i = i0 + q;
      float c = 0.0f, dc = 0.0f;
      if (i < a.n) {
        const pa::fpair r2 = pa::sqdist<DMAX>(a.xs + i * a.d, xp, a.d);
        pa::fpair k, dk;
        if constexpr (DERIV) {
          kernel_and_dl(r2, a.kernel, a.kc, a.dlc, C, k, dk);
        } else {
          k = pa::kernel_entry(r2, a.kernel, a.kc, C);
        }
        const double v = (a.f2 * pa::to_double(k) - pa::to_double(acc[q])) * inv;
        c = static_cast<float>(v);
        if constexpr (DERIV) {
          const double dS = a.f2 * pa::to_double(dk) - pa::to_double(dacc[q]);
          dc = static_cast<float>((dS - v * ddp * 0.5 * inv) * inv);
        }
        double dn = a.dg[i] - static_cast<double>(c) * c;
        if (i == p) dn = 0.0;
        a.dg[i] = dn;
        better(best, besti, dn, i);
      }
      out[q] = c;
      dout[q] = dc;
    }
    store_rows<ROWS>(a.Lt + static_cast<int64_t>(j) * a.n_pad + i0, out);
    if constexpr (DERIV) store_rows<ROWS>(a.Ldt + static_cast<int64_t>(j) * a.n_pad + i0, dout);
  }
  // Block argmax, then the last block picks the next pivot.
  __shared__ double wv[kStepThreads / 32];
  __shared__ long long wi[kStepThreads / 32];
  warp_argmax(best, besti);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    wv[warp] = best;
    wi[warp] = besti;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -INFINITY;
    long long ix = LLONG_MAX;
    for (int w = 0; w < kStepThreads / 32; ++w) better(v, ix, wv[w], wi[w]);
    a.amax_v[blockIdx.x] = v;
    a.amax_i[blockIdx.x] = ix;
  }
  if (!last_block(&S->ticket)) return;
  __shared__ int go_on;
  __shared__ long long next;
  if (warp == 0) {
    double v = -INFINITY;
    long long ix = LLONG_MAX;
    for (unsigned b = lane; b < gridDim.x; b += 32) better(v, ix, a.amax_v[b], a.amax_i[b]);
    warp_argmax(v, ix);
    if (lane == 0) {
      a.piv[j] = p;
      S->rank = j + 1;
      const bool cont = (v > a.tol_abs) && (j + 1 < a.kmax) && ix < a.n;
      S->stop = cont ? 0 : 1;
      S->pivot = cont ? ix : 0;
      S->dp = v;
      go_on = cont ? 1 : 0;
      next = ix;
    }
  }
  __syncthreads();
  if (go_on) {
    double part = 0.0;
    for (int m = threadIdx.x; m <= j; m += blockDim.x) {
      const float lv = a.Lt[static_cast<int64_t>(m) * a.n_pad + next];
      a.prow[m] = lv;
      if constexpr (DERIV) {
        const float dv = a.Ldt[static_cast<int64_t>(m) * a.n_pad + next];
        a.dprow[m] = dv;
        part += static_cast<double>(lv) * dv;
      }
    }
    if constexpr (DERIV) {
      // dd_p of the next pivot, summed in a fixed order.
      __shared__ double red[kStepThreads];
      red[threadIdx.x] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kStepThreads; ++q) t += red[q];
        S->ddp = -2.0 * t;
      }
    }
  }
}

// ------------------------------------------------------------------- Gram --

// Partial sums of L^T L over one chunk of rows, for one 64 x 64 tile pair
// (ta >= tb) of the lower triangle; with TWO, of L^T Bm (Bm = dL/dl) for every
// tile pair (ta, tb), t = ta * tiles + tb.  Dot2 accumulation, renormalised
// per slab.
template <bool TWO>
__global__ void __launch_bounds__(256)
    nys_gram_kernel(const float* __restrict__ Lt, const float* __restrict__ Bm, int64_t n_pad, int r,
                    int64_t rows_per_chunk, int pairs, int tiles, double* gpart) {
  __shared__ __align__(16) float As[kGK][kGT + 4];
  __shared__ __align__(16) float Bs[kGK][kGT + 4];
  const int t = blockIdx.x;
  int ta, tb;
  if constexpr (TWO) {
    ta = t / tiles;
    tb = t - ta * tiles;
  } else {
    ta = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (ta * (ta + 1) / 2 > t) --ta;
    while ((ta + 1) * (ta + 2) / 2 <= t) ++ta;
    tb = t - ta * (ta + 1) / 2;
  }
  const float* Bsrc = TWO ? Bm : Lt;
  const int64_t i_begin = static_cast<int64_t>(blockIdx.y) * rows_per_chunk;
  const int64_t i_end = i_begin + rows_per_chunk < n_pad ? i_begin + rows_per_chunk : n_pad;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  pa::fpair acc[4][4] = {};
  for (int64_t i0 = i_begin; i0 < i_end; i0 += kGK) {
    for (int q = threadIdx.x; q < kGT * (kGK / 4); q += blockDim.x) {
      const int aa = q / (kGK / 4), part = q % (kGK / 4);
      const int ra = ta * kGT + aa, rb = tb * kGT + aa;
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
      if (ra < r) va = *reinterpret_cast<const float4*>(Lt + static_cast<int64_t>(ra) * n_pad + i0 + part * 4);
      if (rb < r) vb = *reinterpret_cast<const float4*>(Bsrc + static_cast<int64_t>(rb) * n_pad + i0 + part * 4);
      As[part * 4 + 0][aa] = va.x;
      As[part * 4 + 1][aa] = va.y;
      As[part * 4 + 2][aa] = va.z;
      As[part * 4 + 3][aa] = va.w;
      Bs[part * 4 + 0][aa] = vb.x;
      Bs[part * 4 + 1][aa] = vb.y;
      Bs[part * 4 + 2][aa] = vb.z;
      Bs[part * 4 + 3][aa] = vb.w;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < kGK; ++ii) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[ii][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[ii][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc_prod(acc[p][q], av[p], bv[q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) renorm(acc[p][q]);
    __syncthreads();
  }
  double* out = gpart + (static_cast<int64_t>(blockIdx.y) * pairs + t) * (kGT * kGT);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(ty * 4 + p) * kGT + tx * 4 + q] = pa::to_double(acc[p][q]);
}

// C[a][b] = sum over chunks (fixed order) + s [a == b] for a >= b; 0 above.
__global__ void nys_gram_reduce_kernel(const double* gpart, int r, int pairs, int chunks, double s,
                                       double* C) {
  const int64_t total = static_cast<int64_t>(r) * r;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int a = static_cast<int>(e / r), b = static_cast<int>(e % r);
    if (b > a) {
      C[e] = 0.0;
      continue;
    }
    const int ta = a / kGT, tb = b / kGT;
    const int t = ta * (ta + 1) / 2 + tb;
    const int64_t off = static_cast<int64_t>(t) * (kGT * kGT) + (a % kGT) * kGT + (b % kGT);
    double v = 0.0;
    for (int ch = 0; ch < chunks; ++ch) v += gpart[static_cast<int64_t>(ch) * pairs * (kGT * kGT) + off];
    C[e] = a == b ? v + s : v;
  }
}

// <C^-1, H> = sum_{a,b < r} Winv[a][b] H[a][b] with H = sum over chunks of the
// TWO Gram partials; per-block FP64 partials in a fixed order, summed by the
// last block into S->tr_wh.
__global__ void nys_trwh_kernel(const double* gpart2, int chunks, int tiles, int r,
                                const double* Winv, double* red, NysState* S) {
  const int64_t total = static_cast<int64_t>(r) * r;
  const int64_t slot = static_cast<int64_t>(tiles) * tiles * (kGT * kGT);
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int a = static_cast<int>(e / r), b = static_cast<int>(e % r);
    const int64_t off = (static_cast<int64_t>(a / kGT) * tiles + b / kGT) * (kGT * kGT) +
                        (a % kGT) * kGT + (b % kGT);
    double h = 0.0;
    for (int ch = 0; ch < chunks; ++ch) h += gpart2[ch * slot + off];
    acc += Winv[e] * h;
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < blockDim.x; ++q) t += sm[q];
    red[blockIdx.x] = t;
  }
  if (!last_block(&S->ticket)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned q = 0; q < gridDim.x; ++q) t += red[q];
    S->tr_wh = t;
  }
}

// log|C| = 2 sum log cdiag and tr(C^-1), one block, fixed order.
__global__ void nys_scalars_kernel(const double* cdiag, const double* Winv, int r, NysState* S) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    a += log(cdiag[j]);
    b += Winv[static_cast<int64_t>(j) * r + j];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < blockDim.x; ++q) {
      ta += s1[q];
      tb += s2[q];
    }
    S->logdet_c = 2.0 * ta;
    S->tr_w = tb;
  }
}

__global__ void nys_terms_kernel(const NysState* S, int64_t n, int r, double s, double f,
                                 double* logdet_m, double* trm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double nr = static_cast<double>(n - r);
  logdet_m[0] = nr * log(s) + S->logdet_c;
  trm[0] = nr / s + S->tr_w;
  trm[1] = (2.0 / f) * (static_cast<double>(r) - s * S->tr_w);
  trm[2] = 2.0 * S->tr_wh;
}

// ------------------------------------------------------------------ probes --

__device__ __forceinline__ uint64_t splitmix64_hash(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Standard normal value of (row i, column c): Box-Muller on two hashed uniforms.
__device__ __forceinline__ double gauss_eps(uint64_t tag, int c, int64_t i) {
  const uint64_t base = tag ^ (static_cast<uint64_t>(c) << 40);
  const uint64_t h1 = splitmix64_hash(base ^ static_cast<uint64_t>(2 * i));
  const uint64_t h2 = splitmix64_hash(base ^ static_cast<uint64_t>(2 * i + 1));
  const double u1 = static_cast<double>((h1 >> 11) + 1) * 0x1.0p-53;
  const double u2 = static_cast<double>(h2 >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

// B[i][col0 + c] = sqrt(s) e2[i][c] (i < n; 0 below), Tp[m][col0 + c] = -e1[m][c]
// as pairs (m < r; every other Tp entry 0), so that the Z kernel with scale 1
// turns B into sqrt(s) e2 + L e1.
__global__ void nys_eps_kernel(const float* eps, uint64_t tag, int64_t n, int64_t n_pad, int r,
                               int p, int col0, int w_pad, double sqrt_s, float* B, float* Tp) {
  const int64_t total = (n_pad + r) * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = e / w_pad;
    const int col = static_cast<int>(e - row * w_pad);
    const int c = col - col0;
    const bool live = c >= 0 && c < p;
    if (row < n_pad) {
      if (!live) continue;
      float v = 0.0f;
      if (row < n) {
        const double g = eps != nullptr ? static_cast<double>(eps[row * p + c]) : gauss_eps(tag, c, row);
        v = static_cast<float>(sqrt_s * g);
      }
      B[row * w_pad + col] = v;
    } else {
      const int64_t m = row - n_pad;
      float v = 0.0f;
      if (live) {
        const int64_t erow = n + m;
        v = eps != nullptr ? eps[erow * p + c] : static_cast<float>(gauss_eps(tag, c, erow));
      }
      Tp[(m * w_pad + col) * 2] = -v;
      Tp[(m * w_pad + col) * 2 + 1] = 0.0f;
    }
  }
}

// ------------------------------------------------------- C's factorisation --

// Right-looking step j of the outer-product Cholesky without scaling:
// a_il -= a_ij a_lj / a_jj for j < l <= i < r (column j itself is read only).
__global__ void nys_chol_step_kernel(double* C, int r, int j, NysState* S) {
  const double ajj = C[static_cast<int64_t>(j) * r + j];
  if (!(ajj > 0.0)) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) S->err = kDevNumeric;
    return;
  }
  if (blockIdx.x > blockIdx.y) return;   // tile entirely above the diagonal
  __shared__ double ci[16], cl[16];
  const int base = j + 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (threadIdx.x < 16) {
    const int i = base + blockIdx.y * 16 + threadIdx.x;
    ci[threadIdx.x] = i < r ? C[static_cast<int64_t>(i) * r + j] : 0.0;
  } else if (threadIdx.x < 32) {
    const int l = base + blockIdx.x * 16 + threadIdx.x - 16;
    cl[threadIdx.x - 16] = l < r ? C[static_cast<int64_t>(l) * r + j] / ajj : 0.0;
  }
  __syncthreads();
  const int i = base + blockIdx.y * 16 + ty, l = base + blockIdx.x * 16 + tx;
  if (i < r && l <= i) C[static_cast<int64_t>(i) * r + l] -= ci[ty] * cl[tx];
}

__global__ void nys_chol_diag_kernel(const double* C, int r, double* cdiag) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < r; j += gridDim.x * blockDim.x)
    cdiag[j] = sqrt(C[static_cast<int64_t>(j) * r + j]);
}

// Factor entries L_C[i][j] = a_ij / sqrt(a_jj) (i >= j), mirrored above the diagonal.
__global__ void nys_chol_scale_kernel(double* C, int r, const double* cdiag) {
  const int64_t total = static_cast<int64_t>(r) * r;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / r), j = static_cast<int>(e % r);
    if (j > i) continue;
    if (i == j) {
      C[e] = cdiag[j];
    } else {
      const double v = C[e] / cdiag[j];
      C[e] = v;
      C[static_cast<int64_t>(j) * r + i] = v;
    }
  }
}

// Column c of C^-1 (= row c, C symmetric): forward substitution L_C y = e_c,
// then back substitution L_C^T x = y, one warp per column, FP64.
__global__ void nys_inverse_kernel(const double* C, int r, double* Winv) {
  extern __shared__ double ysh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kInvWarps + warp;
  if (c >= r) return;
  double* y = ysh + static_cast<int64_t>(warp) * r;
  for (int m = lane; m < c; m += 32) y[m] = 0.0;
  __syncwarp();
  for (int jj = c; jj < r; ++jj) {
    const double* row = C + static_cast<int64_t>(jj) * r;
    double part = 0.0;
    for (int m = c + lane; m < jj; m += 32) part += row[m] * y[m];
    part = warp_sum(part);
    if (lane == 0) y[jj] = ((jj == c ? 1.0 : 0.0) - part) / row[jj];
    __syncwarp();
  }
  for (int jj = r - 1; jj >= 0; --jj) {
    const double* row = C + static_cast<int64_t>(jj) * r;   // upper part: L_C^T row jj
    double part = 0.0;
    for (int m = jj + 1 + lane; m < r; m += 32) part += row[m] * y[m];
    part = warp_sum(part);
    if (lane == 0) y[jj] = (y[jj] - part) / row[jj];
    __syncwarp();
  }
  double* out = Winv + static_cast<int64_t>(c) * r;
  for (int m = lane; m < r; m += 32) out[m] = y[m];
}

// ------------------------------------------------------------------ apply --

// Partial sums of U = L^T V over a chunk of rows: block (x, y, z) covers the
// kLtM columns kLtM y .. of L (rows of Lt) and column group z of V (gw columns
// from c0 = z gw, as column pairs) over chunk x of the rows, in slabs of kGK
// rows staged in shared memory.  Thread t takes column m = t / 4 of L and the
// column pairs k = t % 4 + 4 j, j < NPT, of the group (Dot2 in packed FP32x2,
// renormalised per slab), so every element of L is read once per group.
template <int NPT>
__global__ void __launch_bounds__(256)
    nys_ltv_pk_kernel(const float* __restrict__ Lt, int64_t n_pad, int r,
                      const float* __restrict__ V, int w_pad, int w_live, int gw,
                      int64_t rows_per_chunk, double* upart, const int* active) {
  if (active != nullptr && *active == 0) return;
  constexpr int BC = 8 * NPT;                        // columns staged per slab row
  __shared__ float As[kGK][kLtM + 1];                // L slab, transposed (stride 65: no conflicts)
  __shared__ __align__(16) float Bs[kGK][BC];
  const int m0 = blockIdx.y * kLtM, c0 = blockIdx.z * gw;
  const int cend = min(c0 + gw, w_live);
  const int64_t i_begin = static_cast<int64_t>(blockIdx.x) * rows_per_chunk;
  const int64_t i_end = i_begin + rows_per_chunk < n_pad ? i_begin + rows_per_chunk : n_pad;
  const int tm = threadIdx.x >> 2, tq = threadIdx.x & 3;
  pa2::fp2 acc[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) acc[j] = {pa2::bc(0.0f), pa2::bc(0.0f)};
  for (int64_t i0 = i_begin; i0 < i_end; i0 += kGK) {
    // L slab: kLtM rows of Lt x kGK entries, eight threads per row (coalesced).
    for (int q = threadIdx.x; q < kLtM * (kGK / 4); q += blockDim.x) {
      const int part = q % (kGK / 4), mm = q / (kGK / 4);
      const int m = m0 + mm;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < r) v = *reinterpret_cast<const float4*>(Lt + static_cast<int64_t>(m) * n_pad + i0 + part * 4);
      As[part * 4 + 0][mm] = v.x;
      As[part * 4 + 1][mm] = v.y;
      As[part * 4 + 2][mm] = v.z;
      As[part * 4 + 3][mm] = v.w;
    }
    // V slab: kGK rows x BC columns of the group (zero past its end).
    for (int q = threadIdx.x; q < kGK * (BC / 4); q += blockDim.x) {
      const int ii = q / (BC / 4), h = q % (BC / 4);
      const int c = c0 + h * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < cend) v = *reinterpret_cast<const float4*>(V + (i0 + ii) * w_pad + c);
      *reinterpret_cast<float4*>(&Bs[ii][h * 4]) = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < kGK; ++ii) {
      const float a = As[ii][tm];
#pragma unroll
      for (int j = 0; j < NPT; ++j)
        acc_prod2(acc[j], a, *reinterpret_cast<const float2*>(&Bs[ii][2 * (tq + 4 * j)]));
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j) renorm2(acc[j]);
    __syncthreads();
  }
  const int m = m0 + tm;
  if (m >= r) return;
  double* out = upart + (static_cast<int64_t>(blockIdx.x) * r + m) * w_pad;
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int c = c0 + 2 * (tq + 4 * j);
    if (c < cend) {
      out[c] = pa::to_double(pa2::lane(acc[j], 0));
      out[c + 1] = pa::to_double(pa2::lane(acc[j], 1));
    }
  }
}

// U = the fixed-order sum of the chunks' partial sums; zero in the columns from
// w_live to w_pad (which the partial sums do not cover).
__global__ void nys_u_reduce_kernel(const double* upart, int chunks, int r, int w_pad, int w_live,
                                    double* U, const int* active) {
  if (active != nullptr && *active == 0) return;
  const int64_t total = static_cast<int64_t>(r) * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double v = 0.0;
    if (static_cast<int>(e % w_pad) < w_live)
      for (int ch = 0; ch < chunks; ++ch) v += upart[static_cast<int64_t>(ch) * total + e];
    U[e] = v;
  }
}

// T = C^-1 U (FP64), stored as FP32 pairs; one warp per (row m, 4 columns).
__global__ void nys_wu_kernel(const double* Winv, const double* U, int r, int w_pad, float* Tp,
                              const int* active) {
  if (active != nullptr && *active == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + warp;
  if (m >= r) return;
  const int c0 = blockIdx.y * 4;
  const double* row = Winv + static_cast<int64_t>(m) * r;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = lane; q < r; q += 32) {
    const double wq = row[q];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) acc[cc] += wq * U[static_cast<int64_t>(q) * w_pad + c0 + cc];
  }
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const double t = warp_sum(acc[cc]);
    if (lane == 0) {
      const pa::fpair p = pa::from_double(t);
      float* o = Tp + (static_cast<int64_t>(m) * w_pad + c0 + cc) * 2;
      o[0] = p.hi;
      o[1] = p.lo;
    }
  }
}

// Tp = -U / s as pairs (so that the Z kernel with scale s gives s V + L U).
__global__ void nys_mneg_kernel(const double* U, int r, int w_pad, double inv_s, float* Tp,
                                const int* active) {
  if (active != nullptr && *active == 0) return;
  const int64_t total = static_cast<int64_t>(r) * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const pa::fpair p = pa::from_double(-U[e] * inv_s);
    Tp[2 * e] = p.hi;
    Tp[2 * e + 1] = p.lo;
  }
}

// Z = (V - L T) * scale over column group y (gw columns from c0 = y gw, as
// column pairs); one row per thread, NPZ column pairs per thread (packed FP32x2
// Dot2 with T = thi + tlo: the high part's product exact, the low part's folded
// into the error term), T staged in shared memory kZTile rows at a time as
// (thi, thi, tlo, tlo) per pair; the columns from w_live to w_pad of Z are
// written as zeros.  V and Z may be the same block: each element is read, then
// written, by one thread.
template <int NPZ>
__global__ void __launch_bounds__(256)
    nys_z_pk_kernel(const float* __restrict__ Lt, int64_t n_pad, int64_t n, int r, const float* Tp,
                    const float* V, float* Z, int w_pad, int w_live, int gw, double scale,
                    const int* active) {
  if (active != nullptr && *active == 0) return;
  __shared__ float4 sT[kZTile][NPZ];
  const int c0 = blockIdx.y * gw;
  const int cend = min(c0 + gw, w_live);
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  pa2::fp2 acc[NPZ];
#pragma unroll
  for (int k = 0; k < NPZ; ++k) acc[k] = {pa2::bc(0.0f), pa2::bc(0.0f)};
  for (int mt = 0; mt < r; mt += kZTile) {
    const int mcount = r - mt < kZTile ? r - mt : kZTile;
    __syncthreads();
    for (int q = threadIdx.x; q < kZTile * NPZ; q += blockDim.x) {
      const int mm = q / NPZ, k = q % NPZ;
      const int c = c0 + 2 * k;
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mm < mcount && c < cend) {
        const float4 pr = *reinterpret_cast<const float4*>(Tp + (static_cast<int64_t>(mt + mm) * w_pad + c) * 2);
        t = make_float4(pr.x, pr.z, pr.y, pr.w);
      }
      sT[mm][k] = t;
    }
    __syncthreads();
    if (i < n) {
      const float* col = Lt + static_cast<int64_t>(mt) * n_pad + i;
      int mm = 0;
      for (; mm + kStepBatch <= mcount; mm += kStepBatch) {
        float l[kStepBatch];
#pragma unroll
        for (int u = 0; u < kStepBatch; ++u) l[u] = col[static_cast<int64_t>(mm + u) * n_pad];
#pragma unroll
        for (int u = 0; u < kStepBatch; ++u)
#pragma unroll
          for (int k = 0; k < NPZ; ++k) {
            const float4 t = sT[mm + u][k];
            acc_prod_pair2(acc[k], l[u], make_float2(t.x, t.y), make_float2(t.z, t.w));
          }
      }
      for (; mm < mcount; ++mm) {
        const float l = col[static_cast<int64_t>(mm) * n_pad];
#pragma unroll
        for (int k = 0; k < NPZ; ++k) {
          const float4 t = sT[mm][k];
          acc_prod_pair2(acc[k], l, make_float2(t.x, t.y), make_float2(t.z, t.w));
        }
      }
#pragma unroll
      for (int k = 0; k < NPZ; ++k) renorm2(acc[k]);
    }
  }
  if (i >= n_pad) return;
  if (blockIdx.y == 0)
    for (int c = w_live; c < w_pad; ++c) Z[i * w_pad + c] = 0.0f;
#pragma unroll
  for (int k = 0; k < NPZ; ++k) {
    const int c = c0 + 2 * k;
    if (c >= cend) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float z = 0.0f;
      if (i < n)
        z = static_cast<float>((static_cast<double>(V[i * w_pad + c + h]) -
                                pa::to_double(pa2::lane(acc[k], h))) * scale);
      Z[i * w_pad + c + h] = z;
    }
  }
}

int grid_for(int64_t total, int threads, int cap = 152 * 16) {
  int64_t b = (total + threads - 1) / threads;
  if (b > cap) b = cap;
  return static_cast<int>(b < 1 ? 1 : b);
}

int gram_chunks(int pairs) { return std::max(1, std::min(16, (608 + pairs - 1) / pairs)); }

// Tile slots of the Gram partial sums for any rank up to kmax (chunks x pairs
// is not monotone in the rank).
// Tile slots of the L^T dL/dl partial sums (all tile pairs) for any rank up to kmax.
size_t gram2_slots(int kmax) {
  const int tiles = (kmax + kGT - 1) / kGT;
  size_t most = 0;
  for (int t = 1; t <= tiles; ++t)
    most = std::max(most, static_cast<size_t>(gram_chunks(t * t)) * t * t);
  return most;
}

size_t gram_slots(int kmax) {
  const int tiles = (kmax + kGT - 1) / kGT;
  size_t most = 0;
  for (int t = 1; t <= tiles; ++t) {
    const int pairs = t * (t + 1) / 2;
    most = std::max(most, static_cast<size_t>(gram_chunks(pairs)) * pairs);
  }
  return most;
}

int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct NysCarve {
  char* base;
  size_t off = 0;
  explicit NysCarve(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace

NysWs carve_nys(void* base, int64_t n_pad, int d, int kmax, int w_pad, bool deriv) {
  NysCarve c(base);
  NysWs w{};
  const int step_blocks = static_cast<int>((n_pad + kStepThreads - 1) / kStepThreads);   // most: 1 row per thread
  const int64_t chunks = (n_pad + kLtvChunk - 1) / kLtvChunk;
  w.xs = c.take<float>(static_cast<size_t>(n_pad) * d);
  w.Lt = c.take<float>(static_cast<size_t>(kmax) * n_pad);
  w.dg = c.take<double>(n_pad);
  w.prow = c.take<float>(kmax);
  w.piv = c.take<long long>(kmax);
  w.amax_v = c.take<double>(step_blocks);
  w.amax_i = c.take<long long>(step_blocks);
  w.S = c.take<NysState>(1);
  w.C = c.take<double>(static_cast<size_t>(kmax) * kmax);
  w.cdiag = c.take<double>(kmax);
  w.Winv = c.take<double>(static_cast<size_t>(kmax) * kmax);
  w.gpart = c.take<double>(gram_slots(kmax) * kGT * kGT);
  w.upart = c.take<double>(static_cast<size_t>(chunks) * kmax * w_pad);
  w.U = c.take<double>(static_cast<size_t>(kmax) * w_pad);
  w.Tp = c.take<float>(static_cast<size_t>(kmax) * w_pad * 2);
  w.tred = c.take<double>(kRedCap);
  if (deriv) {
    w.Ldt = c.take<float>(static_cast<size_t>(kmax) * n_pad);
    w.dprow = c.take<float>(kmax);
    w.gpart2 = c.take<double>(gram2_slots(kmax) * kGT * kGT);
    w.U2 = c.take<double>(static_cast<size_t>(kmax) * w_pad);
  }
  w.n_pad = n_pad;
  w.kmax = kmax;
  w.w_pad = w_pad;
  w.w_live = w_pad;
  w.d = d;
  w.deriv = deriv;
  w.bytes = c.off + 256;
  return w;
}

size_t nys_bytes(int64_t n_pad, int d, int kmax, int w_pad, bool deriv) {
  return carve_nys(nullptr, n_pad, d, kmax, w_pad, deriv).bytes;
}

cudaError_t nys_build(const NysWs& W, const NysProblem& P, int kmax, double tol_abs, int* rank,
                      int* dev_err, cudaStream_t st) {
  *rank = 0;
  *dev_err = 0;
  if (kmax < 1 || kmax > W.kmax || P.d > GP_MAX_DIM || P.d != W.d) return cudaErrorInvalidValue;
  const int64_t n_pad = W.n_pad;
  const double f2 = P.f * P.f;
  StageScales sc;
  for (int t = 0; t < GP_MAX_DIM; ++t) sc.v[t] = 1.0f;
  double kl = P.l;
  if (P.ls != nullptr) {
    for (int t = 0; t < P.d; ++t) sc.v[t] = static_cast<float>(1.0 / P.ls[t]);
    kl = 1.0;
  }
  nys_init_kernel<<<grid_for(n_pad, 256), 256, 0, st>>>(P.X, P.n, P.d, sc, n_pad, f2, W.xs, W.dg, W.S);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static pa::ExpConsts consts = [] {
    pa::ExpConsts c;
    pa::make_exp_consts(c);
    return c;
  }();
  StepArgs a{};
  a.xs = W.xs;
  a.n = P.n;
  a.n_pad = n_pad;
  a.d = P.d;
  a.kernel = P.kernel;
  a.kc = pa::kernel_pair_const(P.kernel, kl);
  a.f2 = f2;
  a.tol_abs = tol_abs;
  a.kmax = kmax;
  a.Lt = W.Lt;
  a.dg = W.dg;
  a.prow = W.prow;
  a.piv = W.piv;
  a.amax_v = W.amax_v;
  a.amax_i = W.amax_i;
  a.S = W.S;
  a.Ldt = W.Ldt;
  a.dprow = W.dprow;
  a.dlc = pa::from_double(P.kernel == 0 ? 1.0 / (kl * kl * kl) : 1.0 / kl);
  const bool deriv = W.deriv;
  if (deriv && P.ls != nullptr) return cudaErrorInvalidValue;
  const int wide_blocks =
      static_cast<int>((n_pad + kStepThreads * kStepRowsWide - 1) / (kStepThreads * kStepRowsWide));
  const bool wide = !deriv || wide_blocks >= kStepWideMinBlocks;
  const int blocks = wide ? wide_blocks : static_cast<int>((n_pad + kStepThreads - 1) / kStepThreads);
  const size_t smem = static_cast<size_t>(kmax) * sizeof(float) * (deriv ? 2 : 1);
  for (int j = 0; j < kmax; ++j) {
    if (deriv && wide)
      nys_step_kernel<GP_MAX_DIM, true, kStepRowsWide><<<blocks, kStepThreads, smem, st>>>(a, consts, j);
    else if (deriv)
      nys_step_kernel<GP_MAX_DIM, true, 1><<<blocks, kStepThreads, smem, st>>>(a, consts, j);
    else
      nys_step_kernel<GP_MAX_DIM, false, kStepRowsWide><<<blocks, kStepThreads, smem, st>>>(a, consts, j);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  NysState hs;
  if ((e = cudaMemcpyAsync(&hs, W.S, sizeof hs, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const int r = hs.rank;
  *rank = r;
  if (r < 1) return cudaErrorInvalidValue;
  // C = s I + L^T L.
  const int tiles = (r + kGT - 1) / kGT;
  const int pairs = tiles * (tiles + 1) / 2;
  const int G = gram_chunks(pairs);
  const int64_t rows_per_chunk = round_up64((n_pad + G - 1) / G, kGK);
  nys_gram_kernel<false><<<dim3(pairs, G), 256, 0, st>>>(W.Lt, W.Lt, n_pad, r, rows_per_chunk, pairs,
                                                         tiles, W.gpart);
  count_launch();
  nys_gram_reduce_kernel<<<grid_for(static_cast<int64_t>(r) * r, 256), 256, 0, st>>>(W.gpart, r, pairs,
                                                                                     G, P.s, W.C);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Cholesky factorisation of C, then C^-1.
  for (int j = 0; j + 1 < r; ++j) {
    const int t = (r - j - 1 + 15) / 16;
    nys_chol_step_kernel<<<dim3(t, t), 256, 0, st>>>(W.C, r, j, W.S);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  nys_chol_diag_kernel<<<grid_for(r, 256), 256, 0, st>>>(W.C, r, W.cdiag);
  count_launch();
  nys_chol_scale_kernel<<<grid_for(static_cast<int64_t>(r) * r, 256), 256, 0, st>>>(W.C, r, W.cdiag);
  count_launch();
  const size_t ismem = static_cast<size_t>(kInvWarps) * r * sizeof(double);
  if ((e = cudaFuncSetAttribute(nys_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(ismem))) != cudaSuccess)
    return e;
  nys_inverse_kernel<<<(r + kInvWarps - 1) / kInvWarps, 32 * kInvWarps, ismem, st>>>(W.C, r, W.Winv);
  count_launch();
  nys_scalars_kernel<<<1, 256, 0, st>>>(W.cdiag, W.Winv, r, W.S);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (deriv) {
    // <C^-1, L^T dL/dl>.
    const int t2 = tiles * tiles;
    const int G2 = gram_chunks(t2);
    const int64_t rpc2 = round_up64((n_pad + G2 - 1) / G2, kGK);
    nys_gram_kernel<true><<<dim3(t2, G2), 256, 0, st>>>(W.Lt, W.Ldt, n_pad, r, rpc2, t2, tiles,
                                                        W.gpart2);
    count_launch();
    nys_trwh_kernel<<<grid_for(static_cast<int64_t>(r) * r, 256, kRedCap), 256, 0, st>>>(
        W.gpart2, G2, tiles, r, W.Winv, W.tred, W.S);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpyAsync(&hs, W.S, sizeof hs, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  if (hs.err != 0) {
    *dev_err = hs.err;
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// U = Lm^T V for Lm = L or dL/dl: the tiled partial sums over row chunks (as
// many chunks as keep about four blocks per SM busy, within upart's
// allocation), then their fixed-order sum.
static cudaError_t ltv_into(const NysWs& W, const float* Lm, int rank, const float* V, double* U,
                           const int* active, cudaStream_t st) {
  const int64_t n_pad = W.n_pad;
  const int w_pad = W.w_pad, live = W.w_live;
  // Column groups of at most 2 kLtPairs live columns, as even as multiples of 4 allow.
  const int ng = (live + 2 * kLtPairs - 1) / (2 * kLtPairs);
  const int gw = static_cast<int>(round_up64((live + ng - 1) / ng, 4));
  const int npt = (gw / 2 + 3) / 4;
  const int mt = (rank + kLtM - 1) / kLtM;
  const int64_t max_chunks = (n_pad + kLtvChunk - 1) / kLtvChunk;
  const int64_t G = std::max<int64_t>(1, std::min<int64_t>(max_chunks, (608 + mt * ng - 1) / (mt * ng)));
  const int64_t rpc = round_up64((n_pad + G - 1) / G, kGK);
  const int chunks = static_cast<int>((n_pad + rpc - 1) / rpc);
  const dim3 grid(chunks, mt, ng);
#define GP_LTV_CASE(P)                                                                        \
  case P:                                                                                     \
    nys_ltv_pk_kernel<P><<<grid, 256, 0, st>>>(Lm, n_pad, rank, V, w_pad, live, gw, rpc, W.upart, \
                                               active);                                       \
    break;
  switch (npt) {
    GP_LTV_CASE(1) GP_LTV_CASE(2) GP_LTV_CASE(3) GP_LTV_CASE(4)
    default: GP_LTV_CASE(5)
  }
#undef GP_LTV_CASE
  count_launch();
  nys_u_reduce_kernel<<<grid_for(static_cast<int64_t>(rank) * w_pad, 256), 256, 0, st>>>(
      W.upart, chunks, rank, w_pad, live, U, active);
  count_launch();
  return cudaGetLastError();
}

// Z = (V - L T) * scale with T = W.Tp, in column groups of at most 2 kZPairs
// live columns (as even as pairs allow).
static cudaError_t z_into(const NysWs& W, int rank, int64_t n, const float* V, float* Z, double scale,
                          const int* active, cudaStream_t st) {
  const int64_t n_pad = W.n_pad;
  const int w_pad = W.w_pad, live = W.w_live;
  const int ng = (live + 2 * kZPairs - 1) / (2 * kZPairs);
  const int gw = 2 * ((live / 2 + ng - 1) / ng);
  const dim3 grid(static_cast<unsigned>((n_pad + 255) / 256), static_cast<unsigned>(ng));
#define GP_Z_CASE(P)                                                                          \
  case P:                                                                                     \
    nys_z_pk_kernel<P><<<grid, 256, 0, st>>>(W.Lt, n_pad, n, rank, W.Tp, V, Z, w_pad, live, gw,  \
                                             scale, active);                                  \
    break;
  switch (gw / 2) {
    GP_Z_CASE(1) GP_Z_CASE(2) GP_Z_CASE(3) GP_Z_CASE(4) GP_Z_CASE(5)
    GP_Z_CASE(6) GP_Z_CASE(7) GP_Z_CASE(8) GP_Z_CASE(9)
    default: GP_Z_CASE(10)
  }
#undef GP_Z_CASE
  count_launch();
  return cudaGetLastError();
}

cudaError_t nys_closed_terms(const NysWs& W, int rank, int64_t n, double s, double f,
                             double* logdet_m, double* trm, cudaStream_t st) {
  nys_terms_kernel<<<1, 32, 0, st>>>(W.S, n, rank, s, f, logdet_m, trm);
  count_launch();
  return cudaGetLastError();
}

cudaError_t nys_probes(const NysWs& W, int rank, int64_t n, double s, const float* eps, uint64_t seed,
                       int p, float* B, int col0, cudaStream_t st) {
  const int64_t n_pad = W.n_pad;
  const int w_pad = W.w_pad;
  if (rank < 1 || rank > W.kmax || col0 + p > W.w_live || w_pad % 4 != 0) return cudaErrorInvalidValue;
  const uint64_t tag = seed ^ (1ull << 39);
  nys_eps_kernel<<<grid_for((n_pad + rank) * w_pad, 256), 256, 0, st>>>(
      eps, tag, n, n_pad, rank, p, col0, w_pad, sqrt(s), B, W.Tp);
  count_launch();
  return z_into(W, rank, n, B, B, 1.0, nullptr, st);
}

cudaError_t nys_lt_times(const NysWs& W, int rank, bool deriv_matrix, const float* V, double* U,
                         cudaStream_t st) {
  if (rank < 1 || rank > W.kmax || W.w_pad % 4 != 0 || (deriv_matrix && !W.deriv))
    return cudaErrorInvalidValue;
  return ltv_into(W, deriv_matrix ? W.Ldt : W.Lt, rank, V, U, nullptr, st);
}

cudaError_t nys_apply_m(const NysWs& W, int rank, int64_t n, double s, const float* V, float* Z,
                        const int* active, cudaStream_t st) {
  const int w_pad = W.w_pad;
  if (rank < 1 || rank > W.kmax || w_pad % 4 != 0) return cudaErrorInvalidValue;
  cudaError_t e = ltv_into(W, W.Lt, rank, V, W.U, active, st);
  if (e != cudaSuccess) return e;
  nys_mneg_kernel<<<grid_for(static_cast<int64_t>(rank) * w_pad, 256), 256, 0, st>>>(
      W.U, rank, w_pad, 1.0 / s, W.Tp, active);
  count_launch();
  return z_into(W, rank, n, V, Z, s, active, st);
}

cudaError_t nys_apply(const NysWs& W, int rank, int64_t n, double s, const float* V, float* Z,
                      const int* active, cudaStream_t st) {
  const int w_pad = W.w_pad;
  if (rank < 1 || rank > W.kmax || w_pad % 4 != 0) return cudaErrorInvalidValue;
  cudaError_t e = ltv_into(W, W.Lt, rank, V, W.U, active, st);
  if (e != cudaSuccess) return e;
  nys_wu_kernel<<<dim3((rank + 3) / 4, W.w_live / 4), 128, 0, st>>>(W.Winv, W.U, rank, w_pad, W.Tp,
                                                                     active);
  count_launch();
  return z_into(W, rank, n, V, Z, 1.0 / s, active, st);
}

}  // namespace gp
