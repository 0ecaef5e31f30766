// Fused on-the-fly kernel product on the CUDA cores (FP32).
//
// For a row tile of points x_i and every column tile of points x_j, each entry
// k(|x_i - x_j|) is evaluated once in registers and immediately contracted with
// the V tile, then discarded (the on-the-fly MatVec of §Statement of Need).  The
// derivative entries dk/dl share the same distance evaluation ("kernel matrices
// and its derivatives", §Design and Implementation).
//
// Thread mapping: thread (g, r) owns row r of the CTA's row tile and the TW
// columns [g*TW, (g+1)*TW) of the multivector; all lanes of a warp share g, so
// every shared-memory read of x_j and V[j, :] is a broadcast.  The contraction
// uses packed FP32x2 FMAs.  Sums are blocked: a tile accumulator over kBN
// entries is added into a running sum after each tile, which keeps the FP32
// rounding error at ~eps (sqrt(kBN) + sqrt(n / kBN)) instead of ~eps sqrt(n).
//
// Point and V tiles are staged by the bulk-copy (TMA) engine into a two-stage
// shared-memory ring, each stage completed on its own mbarrier.
#pragma once

#include "gp_internal.cuh"

namespace gp {

template <int DT>
struct DimTraits {
  static constexpr int DP = DT <= 2 ? 2 : ((DT + 3) / 4) * 4;
};

// k and the scaled derivative D' from the scaled squared distance q.
template <int KIND, bool GRAD>
__device__ __forceinline__ void eval_entry(float q, float& kv, float& dv) {
  if constexpr (KIND == GP_KERNEL_GAUSSIAN) {
    kv = dev::ex2_approx(-q);
    if constexpr (GRAD) dv = __fmul_rn(kv, q);
  } else {
    // Explicit roundings so that every variant evaluates bit-identical entries.
    const float a = dev::sqrt_approx(q);
    const float e = dev::ex2_approx(__fmul_rn(a, -1.4426950408889634f));
    kv = __fmaf_rn(a, e, e);
    if constexpr (GRAD) dv = __fmul_rn(a, __fmul_rn(a, e));
  }
}

template <int DT>
__device__ __forceinline__ float sqdist_tile(const float (&xi)[DT], const float* xj) {
  constexpr int DP = DimTraits<DT>::DP;
  float q = 0.f;
  if constexpr (DP == 2) {
    const float2 p = *reinterpret_cast<const float2*>(xj);
    const float d0 = xi[0] - p.x;
    q = d0 * d0;
    if constexpr (DT > 1) {
      const float d1 = xi[1] - p.y;
      q = fmaf(d1, d1, q);
    }
  } else {
#pragma unroll
    for (int t4 = 0; t4 < DP / 4; ++t4) {
      const float4 p = *reinterpret_cast<const float4*>(xj + 4 * t4);
      const float pv[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (4 * t4 + u < DT) {
          const float dd = xi[4 * t4 + u] - pv[u];
          q = fmaf(dd, dd, q);
        }
      }
    }
  }
  return q;
}

template <int KIND, bool GRAD, int DT, int TW>
__global__ void __launch_bounds__(kThreads)
    kmv_simt_kernel(SimtArgs a, int w_pad, int ng, int64_t nr_pad, int jtiles, int jt_per_split) {
  constexpr int DP = DimTraits<DT>::DP;
  constexpr int TW2 = TW / 2;
  static_assert(TW % 4 == 0, "TW must be a multiple of 4");

  if (a.active != nullptr && *a.active == 0) return;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float* sX = reinterpret_cast<float*>(smem_raw + 128);
  float* sV = sX + 2 * kBN * DP;

  const int tid = threadIdx.x;
  const int bm = kBM / ng;
  const int g = tid / bm;
  const int r = tid - g * bm;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * bm + r;
  const int s = blockIdx.y;
  const int jt0 = s * jt_per_split;
  const int jt1 = min(jt0 + jt_per_split, jtiles);
  const int T = jt1 - jt0;

  const uint32_t xbytes = kBN * DP * 4;
  const uint32_t vbytes = kBN * w_pad * 4;

  float xi[DT];
#pragma unroll
  for (int t = 0; t < DT; ++t) xi[t] = a.xr[row * DP + t];

  float2 accK[TW2], runK[TW2];
  float2 accD[GRAD ? TW2 : 1], runD[GRAD ? TW2 : 1];
#pragma unroll
  for (int c = 0; c < TW2; ++c) {
    accK[c] = make_float2(0.f, 0.f);
    runK[c] = make_float2(0.f, 0.f);
    if constexpr (GRAD) {
      accD[c] = make_float2(0.f, 0.f);
      runD[c] = make_float2(0.f, 0.f);
    }
  }

  if (tid == 0) {
    dev::mbar_init(&bars[0], 1);
    dev::mbar_init(&bars[1], 1);
    dev::fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int t, int stage) {
    const int64_t jt = jt0 + t;
    dev::mbar_arrive_expect_tx(&bars[stage], xbytes + vbytes);
    dev::bulk_g2s(sX + stage * kBN * DP, a.xc + jt * kBN * DP, xbytes, &bars[stage]);
    dev::bulk_g2s(sV + stage * kBN * w_pad, a.v + jt * kBN * w_pad, vbytes, &bars[stage]);
  };
  if (tid == 0) {
    if (T > 0) issue(0, 0);
    if (T > 1) issue(1, 1);
  }

  for (int t = 0; t < T; ++t) {
    const int stage = t & 1;
    const uint32_t parity = (t >> 1) & 1;
    const bool ok = dev::mbar_wait(&bars[stage], parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(a.err, kDevTimeout);
        if (t + 1 < T) dev::mbar_wait(&bars[stage ^ 1], ((t + 1) >> 1) & 1);
      }
      return;
    }
    const float* xs = sX + stage * kBN * DP;
    const float* vs = sV + stage * kBN * w_pad + g * TW;
#pragma unroll 2
    for (int jj = 0; jj < kBN; ++jj) {
      const float q = sqdist_tile<DT>(xi, xs + jj * DP);
      float kv, dv;
      eval_entry<KIND, GRAD>(q, kv, dv);
      const float2 kk = make_float2(kv, kv);
      const float2 dd = make_float2(GRAD ? dv : 0.f, GRAD ? dv : 0.f);
      const float4* v4 = reinterpret_cast<const float4*>(vs + jj * w_pad);
#pragma unroll
      for (int c = 0; c < TW / 4; ++c) {
        const float4 v = v4[c];
        const float2 v01 = make_float2(v.x, v.y);
        const float2 v23 = make_float2(v.z, v.w);
        accK[2 * c] = __ffma2_rn(kk, v01, accK[2 * c]);
        accK[2 * c + 1] = __ffma2_rn(kk, v23, accK[2 * c + 1]);
        if constexpr (GRAD) {
          accD[2 * c] = __ffma2_rn(dd, v01, accD[2 * c]);
          accD[2 * c + 1] = __ffma2_rn(dd, v23, accD[2 * c + 1]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < TW2; ++c) {
      runK[c] = __fadd2_rn(runK[c], accK[c]);
      accK[c] = make_float2(0.f, 0.f);
      if constexpr (GRAD) {
        runD[c] = __fadd2_rn(runD[c], accD[c]);
        accD[c] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    if (tid == 0 && t + 2 < T) issue(t + 2, stage);
  }

  const int64_t off = (static_cast<int64_t>(s) * nr_pad + row) * w_pad + g * TW;
  float4* pk = reinterpret_cast<float4*>(a.part_k + off);
#pragma unroll
  for (int c = 0; c < TW / 4; ++c)
    pk[c] = make_float4(runK[2 * c].x, runK[2 * c].y, runK[2 * c + 1].x, runK[2 * c + 1].y);
  if constexpr (GRAD) {
    float4* pd = reinterpret_cast<float4*>(a.part_d + off);
#pragma unroll
    for (int c = 0; c < TW / 4; ++c)
      pd[c] = make_float4(runD[2 * c].x, runD[2 * c].y, runD[2 * c + 1].x, runD[2 * c + 1].y);
  }
}

// Shared-memory bytes of one instantiation.
inline size_t simt_smem_bytes(int dp, int w_pad) {
  return 128 + 2 * static_cast<size_t>(kBN) * dp * 4 + 2 * static_cast<size_t>(kBN) * w_pad * 4;
}

}  // namespace gp
