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
// shared-memory ring, each stage completed on its own mbarrier.  Points are
// stored in tiles of 32, dimension-major within a tile (pt_index), so one
// 16-byte load brings one coordinate of four consecutive points and entries
// are evaluated four at a time in packed FP32x2 arithmetic.
#pragma once

#include "gp_internal.cuh"

namespace gp {

template <int DT>
struct DimTraits {
  static constexpr int DP = DT <= 2 ? 2 : ((DT + 3) / 4) * 4;
};

// k and the scaled derivative D' of two entries from their scaled squared
// distances q, in packed FP32x2 arithmetic (MUFU operations per lane).  Every
// operation is rounded explicitly, so every kernel evaluates bit-identical
// entries.
template <int KIND, bool GRAD>
__device__ __forceinline__ void eval_pair(float2 q, float2& kv, float2& dv) {
  if constexpr (KIND == GP_KERNEL_GAUSSIAN) {
    kv = make_float2(dev::ex2_approx(-q.x), dev::ex2_approx(-q.y));
    if constexpr (GRAD) dv = __fmul2_rn(kv, q);
  } else {
    const float2 a = make_float2(dev::sqrt_approx(q.x), dev::sqrt_approx(q.y));
    const float2 t = __fmul2_rn(a, make_float2(-1.4426950408889634f, -1.4426950408889634f));
    const float2 e = make_float2(dev::ex2_approx(t.x), dev::ex2_approx(t.y));
    kv = __ffma2_rn(a, e, e);
    if constexpr (GRAD) dv = __fmul2_rn(a, __fmul2_rn(a, e));
  }
}

// Scaled squared distances from x_i (each coordinate duplicated into both
// lanes) to the four points j, j+1, j+2, j+3 (j % 4 == 0) of a dimension-major
// point tile xt [dp][32]: (q_j, q_j+1) and (q_j+2, q_j+3).  Difference form:
// d = x_i - x_j as fma(x_j, -1, x_i), q = d0 d0 + d1 d1 + ... left to right.
template <int DT>
__device__ __forceinline__ void sqdist_quad(const float2 (&xi2)[DT], const float* xt, int j,
                                            float2& q01, float2& q23) {
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int t = 0; t < DT; ++t) {
    const float4 p = *reinterpret_cast<const float4*>(xt + t * 32 + j);
    const float2 d01 = __ffma2_rn(make_float2(p.x, p.y), m1, xi2[t]);
    const float2 d23 = __ffma2_rn(make_float2(p.z, p.w), m1, xi2[t]);
    if (t == 0) {
      q01 = __fmul2_rn(d01, d01);
      q23 = __fmul2_rn(d23, d23);
    } else {
      q01 = __ffma2_rn(d01, d01, q01);
      q23 = __ffma2_rn(d23, d23, q23);
    }
  }
}

// Coordinates of the row point i, duplicated into both lanes.
template <int DT>
__device__ __forceinline__ void load_row_point(const float* xr, int64_t i, float2 (&xi2)[DT]) {
  constexpr int DP = DimTraits<DT>::DP;
#pragma unroll
  for (int t = 0; t < DT; ++t) {
    const float v = xr[pt_index(i, t, DP)];
    xi2[t] = make_float2(v, v);
  }
}

// One work item of the product: row tile `row_tile` and j-split `s` of the
// problem `a`, on the calling CTA (shared memory smem_raw).  Returns
// kTileSkipped if the problem's active flag is 0 (nothing touched),
// kTileDone, or kTileTimeout if a bounded wait gave up (the CTA's copies are
// drained, bounded, and *a.err is set).
constexpr int kTileSkipped = 0;
constexpr int kTileDone = 1;
constexpr int kTileTimeout = 2;

template <int KIND, bool GRAD, int DT, int TW>
__device__ __forceinline__ int simt_tile(const SimtArgs& a, int w_pad, int ng, int64_t nr_pad,
                                          int jtiles, int jt_per_split, int row_tile, int s,
                                          unsigned char* smem_raw) {
  constexpr int DP = DimTraits<DT>::DP;
  constexpr int TW2 = TW / 2;
  // Quads of entries per loop iteration: eight let the scheduler overlap one
  // quad's evaluation with another's contraction; fewer for the long distance
  // loops of d > 4, which already give that overlap (and build faster).
  constexpr int kQuadUnroll = DT >= 16 ? 2 : (DT >= 8 ? 4 : 8);
  static_assert(TW % 4 == 0, "TW must be a multiple of 4");

  if (a.active != nullptr && *a.active == 0) return kTileSkipped;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float* sX = reinterpret_cast<float*>(smem_raw + 128);
  float* sV = sX + 2 * kBN * DP;

  const int tid = threadIdx.x;
  const int bm = kBM / ng;
  const int g = tid / bm;
  const int r = tid - g * bm;
  const int64_t row = static_cast<int64_t>(row_tile) * bm + r;
  const int jt0 = s * jt_per_split;
  const int jt1 = min(jt0 + jt_per_split, jtiles);
  const int T = jt1 - jt0;

  const uint32_t xbytes = kBN * DP * 4;
  const uint32_t vbytes = kBN * w_pad * 4;

  float2 xi2[DT];
  load_row_point<DT>(a.xr, row, xi2);

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
      // Before the CTA exits, wait (bounded) for both copies it may still have
      // in flight: tile t's (the one that timed out) and tile t+1's.
      if (tid == 0) {
        atomicExch(a.err, kDevTimeout);
        dev::mbar_wait(&bars[stage], parity);
        if (t + 1 < T) dev::mbar_wait(&bars[stage ^ 1], ((t + 1) >> 1) & 1);
      }
      return kTileTimeout;
    }
    const float* xs = sX + stage * kBN * DP;
    const float* vs = sV + stage * kBN * w_pad + g * TW;
#pragma unroll kQuadUnroll
    for (int jj = 0; jj < kBN; jj += 4) {
      float2 q01, q23;
      sqdist_quad<DT>(xi2, xs + (jj >> 5) * (32 * DP), jj & 31, q01, q23);
      float2 k01, d01 = make_float2(0.f, 0.f), k23, d23 = make_float2(0.f, 0.f);
      eval_pair<KIND, GRAD>(q01, k01, d01);
      eval_pair<KIND, GRAD>(q23, k23, d23);
      const float kq[4] = {k01.x, k01.y, k23.x, k23.y};
      const float dq[4] = {d01.x, d01.y, d23.x, d23.y};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 kk = make_float2(kq[u], kq[u]);
        const float2 dd = make_float2(dq[u], dq[u]);
        const float4* v4 = reinterpret_cast<const float4*>(vs + (jj + u) * w_pad);
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
  return kTileDone;
}

template <int KIND, bool GRAD, int DT, int TW>
__global__ void __launch_bounds__(kThreads)
    kmv_simt_kernel(SimtArgs a, int w_pad, int ng, int64_t nr_pad, int jtiles, int jt_per_split) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  simt_tile<KIND, GRAD, DT, TW>(a, w_pad, ng, nr_pad, jtiles, jt_per_split, blockIdx.x, blockIdx.y,
                                smem_raw);
}

// The product of several problems in one persistent launch: every CTA takes
// work items (problem, row tile, j-split) from a global counter until none is
// left, so the tiles of all the problems share the SMs.  Each item writes its
// own partial-sum slot, so the result does not depend on which CTA ran it.
// The problems share the instantiation (kernel, grad, dimension template, TW)
// and the padded width; the table is a kernel parameter.
template <int KIND, bool GRAD, int DT, int TW>
__global__ void __launch_bounds__(kThreads)
    kmv_simt_group_kernel(const __grid_constant__ SimtGroup G, int w_pad, int ng) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int item_s;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(G.counter, 1);
    __syncthreads();
    const int item = item_s;
    if (item >= G.total_items) return;
    int k = 0;
    while (k + 1 < G.count && G.e[k + 1].item0 <= item) ++k;
    const SimtGroupEntry& e = G.e[k];
    const int local = item - e.item0;
    const int row_tile = local % e.row_tiles;
    const int split = local / e.row_tiles;
    const int st = simt_tile<KIND, GRAD, DT, TW>(e.a, w_pad, ng, e.nr_pad, e.jtiles,
                                                 e.jt_per_split, row_tile, split, smem_raw);
    // A timed-out item may leave a copy in flight: this CTA stops (the
    // problem's error word is set; the other CTAs finish the other items).
    if (st == kTileTimeout) return;
    // Every thread is past the item (it has read item_s, and its barriers are
    // idle); a finished item's barriers are invalidated so that the next item
    // initialises them afresh.
    __syncthreads();
    if (st == kTileDone && threadIdx.x == 0) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(dev::smem_addr(&bars[0])) : "memory");
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(dev::smem_addr(&bars[1])) : "memory");
    }
  }
}

// Shared-memory bytes of one instantiation.
inline size_t simt_smem_bytes(int dp, int w_pad) {
  return 128 + 2 * static_cast<size_t>(kBN) * dp * 4 + 2 * static_cast<size_t>(kBN) * w_pad * 4;
}

}  // namespace gp
