// Shared pieces of the tensor-core (tcgen05) product: operand modes, the
// K-major core-matrix geometry (8 rows x 16 bytes per core matrix, no swizzle),
// shared- and tensor-memory descriptors, and the PTX wrappers for tcgen05.mma,
// commit, fences, tensor-memory loads and stores.
#pragma once

#include <cuda_bf16.h>

#include "kmv_simt.cuh"
#include "kmv_tc.cuh"

namespace gp {

constexpr int kTcM = 128;        // rows per CTA = MMA M
constexpr int kTcBK = 32;        // points per staged point tile; the widest MMA tile
constexpr int kTcEvalThreads = 256;  // eval warps 0-7: two threads per row
constexpr int kTcThreads = 288;      // + one control warp (copies and MMA issue)
constexpr int kTcBStages = 5;
constexpr int kTcAStages = 2;
constexpr int kTcNumBars = 2 * kTcBStages + 2 * kTcAStages + 1;
static_assert(kTcNumBars * 8 + 8 <= 128, "barriers, tmem holder and abort flag share 128 bytes");
constexpr int kTcFlushCols = 512;  // columns j per accumulation block

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

// Columns j per tile (the MMA K extent of a tile): 32, or 16 for split TF32,
// whose 4-byte hi and lo A operands would otherwise fill 128 KB of shared
// memory per CTA and allow only one CTA per SM.
constexpr int tc_tile_cols(int mode) { return mode == kTcTF32x3 ? 16 : 32; }

// Geometry shared by host and device.
template <int MODE>
struct TcGeom {
  static constexpr int ES = TcTraits<MODE>::ES;
  static constexpr int BK = tc_tile_cols(MODE);       // columns j per tile
  static constexpr int FLUSH = kTcFlushCols / BK;     // tiles per accumulation block
  static constexpr int EPC = 16 / ES;                 // elements per 16-byte core-matrix row
  static constexpr int CK = BK / EPC;                 // core matrices along K per tile
  static constexpr uint32_t SBO = CK * 128;           // bytes between 8-row groups
  static constexpr uint32_t LBO = 128;                // bytes between K-adjacent core matrices
  static constexpr int KSTEPS = CK / 2;               // MMAs (32 bytes of K each) per tile
  static constexpr uint32_t A_BYTES = (kTcM / 8) * SBO;
};

// Split BF16 can keep the A operand (the evaluated kernel tile) in tensor
// memory instead of shared memory: each eval thread writes its row's entries
// with tcgen05.st, two BF16 values per 32-bit column (the lower K index in the
// low half), and the MMA reads A from there, which removes the core-matrix
// shared-memory stores of A.  It costs 128 tensor-memory columns per CTA (two
// stages x K and D x hi and lo x 16), so the host takes it per launch only
// where it keeps as many CTAs resident as the shared-memory form (measured at
// n = 1e5, w = 32 with the gradient: 8.22 ms against 8.88).  Plain BF16 (three
// CTAs per SM with A in shared memory: 5.83 ms, against 6.80 with A in tensor
// memory and two CTAs) and the TF32 modes (4-byte elements) keep A in shared
// memory.
template <int MODE>
struct TcATmem {
  static constexpr bool ON = MODE == kTcBF16x3;
  static constexpr int COLS = TcGeom<MODE>::BK / 2;   // columns per A matrix per stage
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

// A in tensor memory: tcgen05.mma reads A from [atmem] (M rows = lanes 0..127).
template <int MODE>
__device__ __forceinline__ void mma_ts(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t acc) {
  static_assert(TcTraits<MODE>::FMT == 1, "A from tensor memory: BF16 modes only");
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtmem),
      "r"(atmem), "l"(bdesc), "r"(idesc), "r"(acc));
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

__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Store 16 bytes of one operand row (EPC entries, as EPC / 2 pairs) at `off` of
// the hi matrix and, when SPLIT, the rounded remainder at `off` of the lo matrix
// (generic proxy).  The remainder v - hi is formed as fma(hi, -1, v) in packed
// FP32x2, which rounds like the subtraction.
template <int MODE, bool SPLIT>
__device__ __forceinline__ void store_group(unsigned char* hi, unsigned char* lo, uint32_t off,
                                            const float2 (&v)[8 / TcTraits<MODE>::ES]) {
  const float2 m1 = make_float2(-1.f, -1.f);
  if constexpr (TcTraits<MODE>::FMT == 1) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const __nv_bfloat162 p = __floats2bfloat162_rn(v[u].x, v[u].y);
      h[u] = *reinterpret_cast<const uint32_t*>(&p);
      if constexpr (SPLIT) {
        const float2 r = __ffma2_rn(__bfloat1622float2(p), m1, v[u]);
        const __nv_bfloat162 q = __floats2bfloat162_rn(r.x, r.y);
        l[u] = *reinterpret_cast<const uint32_t*>(&q);
      }
    }
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    if constexpr (SPLIT) *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  } else {
    uint32_t h[4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      h[2 * u] = to_tf32(v[u].x);
      h[2 * u + 1] = to_tf32(v[u].y);
    }
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    if constexpr (SPLIT) {
      uint32_t l[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 hv = make_float2(__uint_as_float(h[2 * u]), __uint_as_float(h[2 * u + 1]));
        const float2 r = __ffma2_rn(hv, m1, v[u]);
        l[2 * u] = to_tf32(r.x);
        l[2 * u + 1] = to_tf32(r.y);
      }
      *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

// BF16 packing of 8 entries (4 pairs) into 4 words of hi and, when SPLIT, 4
// words of the rounded remainder lo (the arithmetic of store_group's BF16 path).
template <bool SPLIT>
__device__ __forceinline__ void pack_bf16(const float2 (&v)[4], uint32_t* h, uint32_t* l) {
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(v[u].x, v[u].y);
    h[u] = *reinterpret_cast<const uint32_t*>(&p);
    if constexpr (SPLIT) {
      const float2 r = __ffma2_rn(__bfloat1622float2(p), m1, v[u]);
      const __nv_bfloat162 q = __floats2bfloat162_rn(r.x, r.y);
      l[u] = *reinterpret_cast<const uint32_t*>(&q);
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
__host__ __device__ inline TcSmem tc_smem(int n, bool grad, int nbs, bool atm = false) {
  using G = TcGeom<MODE>;
  constexpr int DP = DimTraits<DT>::DP;
  TcSmem s;
  s.xbytes = kTcBK * DP * 4;   // the 32-point tile holding the tile's points
  s.bbytes = static_cast<uint32_t>(n / 8) * G::SBO;
  s.abytes = G::A_BYTES;
  s.bars = 0;                                 // kTcNumBars mbarriers, tmem holder, abort flag
  s.sx = 128;
  s.sb = s.sx + ((nbs * s.xbytes + 127) / 128) * 128;
  s.sa = s.sb + nbs * TcTraits<MODE>::NSB * s.bbytes;
  s.total = s.sa + ((TcATmem<MODE>::ON && atm)
                         ? 0u
                         : kTcAStages * (grad ? 2 : 1) * TcTraits<MODE>::NSA * s.abytes);
  return s;
}

// Tensor-memory columns: accumulators [0, NMAT*n), running sums [NMAT*n,
// 2*NMAT*n), then (BF16 modes) the A stages, kTcAStages x NMAT x NSA matrices
// of TcATmem::COLS columns.
template <int MODE>
__host__ __device__ inline uint32_t tc_tmem_cols(int n, bool grad, bool atm = false) {
  const int nmat = grad ? 2 : 1;
  int need = 2 * nmat * n;
  if (TcATmem<MODE>::ON && atm)
    need += kTcAStages * nmat * TcTraits<MODE>::NSA * TcATmem<MODE>::COLS;
  uint32_t c = 32;
  while (c < static_cast<uint32_t>(need)) c <<= 1;
  return c;
}


}  // namespace gp
