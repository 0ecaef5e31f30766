// The on-the-fly product with the K-tile x V-tile contraction on the fifth-
// generation tensor cores (tcgen05, sm_103a).
//
// One CTA owns 128 rows (points x_i, the MMA M dimension) and walks the columns
// j in tiles of kTcBK points; two threads share each row, each evaluating half
// of the tile's columns.  Per tile:
//   1. the bulk-copy (TMA) engine brings the tile's points and its slice of V,
//      already laid out as the MMA B operand, into a 3-stage shared ring;
//   2. the threads evaluate k(x_i, x_j) (and dk/dl) in registers and write
//      them, rounded to the operand type, into a 2-stage shared A tile in the
//      K-major core-matrix layout (8 rows x 16 bytes per core matrix, no
//      swizzle);
//   3. one thread issues tcgen05.mma: D_K += A_K B, D_D += A_D B with FP32
//      accumulation in tensor memory; tcgen05.commit then arrives on an
//      mbarrier that frees the tile's A and B buffers.
// Kernel entries never leave the SM (the on-the-fly MatVec of §Statement of
// Need; the derivative shares the distance evaluation).
//
// Blocked accumulation: the tensor-core accumulator restarts every kTcFlush
// tiles, after its block sum has been added (FP32, by the threads) into a
// running sum that also lives in tensor memory.  Accumulation chains therefore
// stay kTcFlush * kTcBK long, which keeps the split-operand modes at FP32-level
// accuracy for any n.
//
// Every mbarrier wait is bounded; on a timeout the CTA records kDevTimeout,
// waits (bounded) for its own copies and MMAs in flight, frees its tensor
// memory and returns.
#pragma once

#include <cuda_bf16.h>

#include "kmv_simt.cuh"
#include "kmv_tc.cuh"

namespace gp {

constexpr int kTcM = 128;        // rows per CTA = MMA M
constexpr int kTcBK = 32;        // points j per tile = MMA K extent per tile
constexpr int kTcThreads = 256;  // two threads per row
constexpr int kTcBStages = 3;
constexpr int kTcAStages = 2;
constexpr int kTcFlush = 16;     // tiles per accumulation block

// NSA / NSB: parts the A (kernel tile) and B (V tile) operands are split into
// (hi, or hi + rounded remainder lo); NPROD: MMAs per K-step and accumulator.
//   TF32:   A tf32,          B tf32          -> A B
//   BF16:   A bf16,          B bf16 hi + lo  -> A B_hi + A B_lo
//   TF32x3: A tf32 hi + lo,  B tf32 hi + lo  -> A_hi B_hi + A_hi B_lo + A_lo B_hi
//   BF16x3: A bf16 hi + lo,  B bf16 hi + lo  -> the same three products
template <int MODE>
struct TcTraits;
template <>
struct TcTraits<kTcTF32> {
  static constexpr int ES = 4, NSA = 1, NSB = 1, NPROD = 1;
  static constexpr uint32_t FMT = 2;  // instruction-descriptor operand format: TF32
};
template <>
struct TcTraits<kTcBF16> {
  static constexpr int ES = 2, NSA = 1, NSB = 2, NPROD = 2;
  static constexpr uint32_t FMT = 1;  // BF16
};
template <>
struct TcTraits<kTcTF32x3> {
  static constexpr int ES = 4, NSA = 2, NSB = 2, NPROD = 3;
  static constexpr uint32_t FMT = 2;
};
template <>
struct TcTraits<kTcBF16x3> {
  static constexpr int ES = 2, NSA = 2, NSB = 2, NPROD = 3;
  static constexpr uint32_t FMT = 1;
};

// Geometry shared by host and device.
template <int MODE>
struct TcGeom {
  static constexpr int ES = TcTraits<MODE>::ES;
  static constexpr int EPC = 16 / ES;                 // elements per 16-byte core-matrix row
  static constexpr int CK = kTcBK / EPC;              // core matrices along K per tile
  static constexpr uint32_t SBO = CK * 128;           // bytes between 8-row groups
  static constexpr uint32_t LBO = 128;                // bytes between K-adjacent core matrices
  static constexpr int KSTEPS = CK / 2;               // MMAs (32 bytes of K each) per tile
  static constexpr uint32_t A_BYTES = (kTcM / 8) * SBO;
};

namespace tc {

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version of tcgen05
  return d;                             // base offset 0, layout: no swizzle
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t acc) {
  if constexpr (TcTraits<MODE>::FMT == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          dev::smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]));
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Store 16 bytes of one operand row (EPC entries) at `off` of the hi matrix and,
// when SPLIT, the rounded remainder at `off` of the lo matrix (generic proxy).
template <int MODE, bool SPLIT>
__device__ __forceinline__ void store_group(unsigned char* hi, unsigned char* lo, uint32_t off,
                                            const float (&v)[16 / TcTraits<MODE>::ES]) {
  if constexpr (TcTraits<MODE>::FMT == 1) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
      h[u] = *reinterpret_cast<const uint32_t*>(&p);
      if constexpr (SPLIT) {
        const float2 back = __bfloat1622float2(p);
        const __nv_bfloat162 r = __floats2bfloat162_rn(v[2 * u] - back.x, v[2 * u + 1] - back.y);
        l[u] = *reinterpret_cast<const uint32_t*>(&r);
      }
    }
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    if constexpr (SPLIT) *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  } else {
    uint32_t h[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) h[u] = to_tf32(v[u]);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    if constexpr (SPLIT) {
      uint32_t l[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) l[u] = to_tf32(v[u] - __uint_as_float(h[u]));
      *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

}  // namespace tc

// Shared-memory plan of one launch (host and device agree on it).
struct TcSmem {
  uint32_t bars, sx, sb, sa, total;
  uint32_t xbytes, bbytes, abytes;  // per stage / per matrix
};

template <int MODE, int DT>
__host__ __device__ inline TcSmem tc_smem(int n, bool grad) {
  using G = TcGeom<MODE>;
  constexpr int DP = DimTraits<DT>::DP;
  TcSmem s;
  s.xbytes = kTcBK * DP * 4;
  s.bbytes = static_cast<uint32_t>(n / 8) * G::SBO;
  s.abytes = G::A_BYTES;
  s.bars = 0;                                 // 5 mbarriers, tmem holder, abort flag
  s.sx = 128;
  s.sb = s.sx + ((kTcBStages * s.xbytes + 127) / 128) * 128;
  s.sa = s.sb + kTcBStages * TcTraits<MODE>::NSB * s.bbytes;
  s.total = s.sa + kTcAStages * (grad ? 2 : 1) * TcTraits<MODE>::NSA * s.abytes;
  return s;
}

// Tensor-memory columns: accumulators [0, NMAT*n) and running sums [NMAT*n, 2*NMAT*n).
__host__ __device__ inline uint32_t tc_tmem_cols(int n, bool grad) {
  const int need = 2 * (grad ? 2 : 1) * n;
  uint32_t c = 32;
  while (c < static_cast<uint32_t>(need)) c <<= 1;
  return c;
}

template <int KIND, bool GRAD, int DT, int MODE>
__global__ void __launch_bounds__(kTcThreads)
    kmv_tc_kernel(TcArgs a, int n_cols, int64_t nr_pad, int jtiles, int jt_per_split,
                  uint32_t idesc, uint32_t tmem_cols) {
  using G = TcGeom<MODE>;
  constexpr int DP = DimTraits<DT>::DP;
  constexpr int NSA = TcTraits<MODE>::NSA;
  constexpr int NSB = TcTraits<MODE>::NSB;
  constexpr int NPROD = TcTraits<MODE>::NPROD;
  constexpr int EPC = G::EPC;
  constexpr int NMAT = GRAD ? 2 : 1;
  constexpr int HALF_CK = G::CK / 2;

  if (a.active != nullptr && *a.active == 0) return;

  extern __shared__ __align__(1024) unsigned char smem[];
  const TcSmem L = tc_smem<MODE, DT>(n_cols, GRAD);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);  // [kTcBStages]
  uint64_t* mmad = full + kTcBStages;                            // [kTcAStages]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mmad + kTcAStages);
  int* abort_s = reinterpret_cast<int*>(tmem_holder + 1);
  float* sX = reinterpret_cast<float*>(smem + L.sx);
  unsigned char* sB = smem + L.sb;
  unsigned char* sA = smem + L.sa;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int m = tid & (kTcM - 1);        // row within the tile
  const int half = tid >> 7;             // which half of the tile's columns
  const int quad = warp & 3;             // tensor-memory lane quadrant of this warp
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kTcM + m;
  const int s = blockIdx.y;
  const int jt0 = s * jt_per_split;
  const int jt1 = min(jt0 + jt_per_split, jtiles);
  const int T = jt1 - jt0;
  const int acc_cols = NMAT * n_cols;    // accumulator columns = running-sum columns

  float xi[DT];
#pragma unroll
  for (int t = 0; t < DT; ++t) xi[t] = a.xr[row * DP + t];

  if (tid == 0) {
    for (int i = 0; i < kTcBStages + kTcAStages; ++i) dev::mbar_init(&full[i], 1);
    *abort_s = 0;
    dev::fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     dev::smem_addr(tmem_holder)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_holder;
  const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;

  // Zero the running sums: warp (quad, half) clears 16-column chunks c % 2 == half.
  {
    uint32_t z[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) z[u] = 0u;
    for (int c0 = 16 * half; c0 < acc_cols; c0 += 32)
      tc::st16(tmem + lane_base + static_cast<uint32_t>(acc_cols + c0), z);
    tc::wait_st();
  }

  // Running sum += accumulator, 16-column chunks split between the halves.
  auto fold = [&]() {
    for (int c0 = 16 * half; c0 < acc_cols; c0 += 32) {
      uint32_t r[16], u[16];
      tc::ld16(tmem + lane_base + static_cast<uint32_t>(c0), r);
      tc::ld16(tmem + lane_base + static_cast<uint32_t>(acc_cols + c0), u);
      tc::wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q)
        u[q] = __float_as_uint(__uint_as_float(u[q]) + __uint_as_float(r[q]));
      tc::st16(tmem + lane_base + static_cast<uint32_t>(acc_cols + c0), u);
    }
    tc::wait_st();
  };

  int issued = 0;       // tiles whose copies were issued (thread 0)
  int committed = -1;   // last tile whose MMAs were committed (thread 0)
  auto issue_copy = [&](int t) {
    const int st = t % kTcBStages;
    const int64_t jt = jt0 + t;
    dev::mbar_arrive_expect_tx(&full[st], L.xbytes + NSB * L.bbytes);
    dev::bulk_g2s(sX + st * (L.xbytes / 4), a.xc + jt * kTcBK * DP, L.xbytes, &full[st]);
    const unsigned char* vsrc = static_cast<const unsigned char*>(a.vt) + jt * NSB * L.bbytes;
    dev::bulk_g2s(sB + st * NSB * L.bbytes, vsrc, NSB * L.bbytes, &full[st]);
  };
  if (tid == 0) {
    for (int t = 0; t < 2 && t < T; ++t) issue_copy(t);
    issued = T < 2 ? T : 2;
  }

  bool bad = false;
  for (int t = 0; t < T; ++t) {
    const int bs = t % kTcBStages;
    const int as = t % kTcAStages;
    const bool fold_now = (t > 0) && (t % kTcFlush == 0);
    bool ok = dev::mbar_wait(&full[bs], (t / kTcBStages) & 1);
    if (ok && t >= kTcAStages) ok = dev::mbar_wait(&mmad[as], ((t - kTcAStages) / kTcAStages) & 1);
    if (ok && fold_now) ok = dev::mbar_wait(&mmad[(t - 1) % kTcAStages], ((t - 1) / kTcAStages) & 1);
    if (__syncthreads_or(!ok || *abort_s != 0)) {
      bad = true;
      break;
    }
    if (fold_now) {
      tc::fence_after();
      fold();
    }
    // Evaluate this thread's half of the row's entries into the A buffers.
    const float* xs = sX + bs * (L.xbytes / 4);
    unsigned char* aK = sA + (as * NMAT * NSA) * L.abytes;
    unsigned char* aD = aK + NSA * L.abytes;
    const uint32_t rowoff = static_cast<uint32_t>(m >> 3) * G::SBO + static_cast<uint32_t>(m & 7) * 16;
#pragma unroll
    for (int kh = 0; kh < HALF_CK; ++kh) {
      const int kg = half * HALF_CK + kh;
      float kv[EPC], dv[EPC];
#pragma unroll
      for (int u = 0; u < EPC; ++u) {
        const float q = sqdist_tile<DT>(xi, xs + (kg * EPC + u) * DP);
        float k1, d1 = 0.f;
        eval_entry<KIND, GRAD>(q, k1, d1);
        kv[u] = k1;
        dv[u] = d1;
      }
      const uint32_t off = rowoff + static_cast<uint32_t>(kg) * G::LBO;
      tc::store_group<MODE, (NSA == 2)>(aK, aK + L.abytes, off, kv);
      if constexpr (GRAD) tc::store_group<MODE, (NSA == 2)>(aD, aD + L.abytes, off, dv);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      const uint32_t a0 = dev::smem_addr(aK);
      const uint32_t b0 = dev::smem_addr(sB + bs * NSB * L.bbytes);
      uint32_t acc = (t % kTcFlush == 0) ? 0u : 1u;   // a block starts from zero
#pragma unroll
      for (int ks = 0; ks < G::KSTEPS; ++ks) {
        // One MMA consumes two K-adjacent core matrices (32 bytes of K).
        const uint32_t ko = static_cast<uint32_t>(ks) * 2 * G::LBO;
        // Products (A part, B part): (hi, hi), then (hi, lo), then (lo, hi).
#pragma unroll
        for (int pr = 0; pr < NPROD; ++pr) {
          const uint32_t am = (pr == 2) ? 1u : 0u;
          const uint32_t bm = (pr == 1) ? 1u : 0u;
          const uint64_t bdesc = tc::smem_desc(b0 + bm * L.bbytes + ko, G::LBO, G::SBO);
          const uint64_t adk = tc::smem_desc(a0 + am * L.abytes + ko, G::LBO, G::SBO);
          tc::mma<MODE>(tmem, adk, bdesc, idesc, acc);
          if constexpr (GRAD) {
            const uint64_t add = tc::smem_desc(a0 + (NSA + am) * L.abytes + ko, G::LBO, G::SBO);
            tc::mma<MODE>(tmem + static_cast<uint32_t>(n_cols), add, bdesc, idesc, acc);
          }
          acc = 1u;
        }
      }
      tc::commit(&mmad[as]);
      committed = t;
      // Refill the B stage that tile t-1 used, once its MMAs are done.
      if (issued < T) {
        bool fr = true;
        if (t >= 1) fr = dev::mbar_wait(&mmad[(t - 1) % kTcAStages], ((t - 1) / kTcAStages) & 1);
        if (fr) {
          issue_copy(issued);
          ++issued;
        } else {
          *abort_s = 1;
        }
      }
    }
  }

  if (!bad) {
    // Wait for the last tile's MMAs (and, by order, all earlier ones).
    bool ok = true;
    if (T > 0) ok = dev::mbar_wait(&mmad[(T - 1) % kTcAStages], ((T - 1) / kTcAStages) & 1);
    if (__syncthreads_or(!ok)) bad = true;
  }
  if (bad) {
    if (tid == 0) {
      atomicExch(a.err, kDevTimeout);
      if (committed >= 0)
        dev::mbar_wait(&mmad[committed % kTcAStages], (committed / kTcAStages) & 1);
      // Copies issued but not consumed: wait for their stages (bounded).
      for (int t = (committed >= 0 ? committed + 1 : 0); t < issued; ++t)
        dev::mbar_wait(&full[t % kTcBStages], (t / kTcBStages) & 1);
    }
  } else {
    tc::fence_after();
    // Output = running sum + last block's accumulator.
    const int64_t off = (static_cast<int64_t>(s) * nr_pad + row) * n_cols;
    for (int c0 = 16 * half; c0 < acc_cols; c0 += 32) {
      uint32_t r[16], u[16];
      tc::ld16(tmem + lane_base + static_cast<uint32_t>(c0), r);
      tc::ld16(tmem + lane_base + static_cast<uint32_t>(acc_cols + c0), u);
      tc::wait_ld();
      float* base = (c0 < n_cols) ? (a.part_k + off + c0) : (a.part_d + off + (c0 - n_cols));
      float4* dst = reinterpret_cast<float4*>(base);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        dst[q] = make_float4(__uint_as_float(u[4 * q]) + __uint_as_float(r[4 * q]),
                             __uint_as_float(u[4 * q + 1]) + __uint_as_float(r[4 * q + 1]),
                             __uint_as_float(u[4 * q + 2]) + __uint_as_float(r[4 * q + 2]),
                             __uint_as_float(u[4 * q + 3]) + __uint_as_float(r[4 * q + 3]));
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

}  // namespace gp
