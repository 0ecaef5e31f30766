// The on-the-fly product with the K-tile x V-tile contraction on the fifth-
// generation tensor cores (tcgen05, sm_103a), warp-specialised.
//
// One CTA owns 128 rows (points x_i, the MMA M dimension) and walks the columns
// j in tiles of G::BK points (32, or 16 for split TF32).
//   * Control warp (warp 8, lane 0): issues the bulk (TMA) copies of each
//     tile's points and of its slice of V, already laid out as the MMA B
//     operand, into a shared ring of up to kTcBStages stages (as many as fit),
//     and issues the tile's tcgen05.mma instructions D_K += A_K B,
//     D_D += A_D B (FP32 accumulation in tensor memory) from descriptors
//     precomputed for stage 0, then tcgen05.commit to the barriers that free
//     the buffers.  (A second issuing warp for D was measured slower.)
//   * Eval warps 0-7 (two threads per row, each half of the tile's columns):
//     evaluate k(x_i, x_j) and dk/dl in registers and write them, rounded to
//     the operand type, into a 2-stage A buffer in the K-major core-matrix
//     layout, then arrive on that stage's "full" barrier.
// The two roles meet only through mbarriers, so the eval warps keep evaluating
// while earlier tiles are in the tensor cores.  Kernel entries never leave the
// SM (the on-the-fly MatVec of §Statement of Need; the derivative shares the
// distance evaluation).
//
// Blocked accumulation: the accumulator restarts every G::FLUSH tiles after the
// eval warps have added its block sum (FP32) into a running sum kept in tensor
// memory, so accumulation chains stay kTcFlushCols = 512 columns long.
//
// Every mbarrier wait is bounded (and polls a shared abort flag); on a timeout
// the CTA records kDevTimeout, waits (bounded) for its own copies and MMAs in
// flight, frees its tensor memory and returns.
#pragma once

#include "kmv_tc_common.cuh"

namespace gp {

namespace tc {

// Bounded wait that also gives up once another thread has set *abort_s.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, const int* abort_s) {
  const uint32_t addr = dev::smem_addr(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023) == 1023 && *reinterpret_cast<const volatile int*>(abort_s) != 0) return false;
  }
  return false;
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(dev::smem_addr(bar)) : "memory");
}

}  // namespace tc

template <int KIND, bool GRAD, int DT, int MODE, bool ATM_T>
// Plain BF16 needs little shared memory, so it can keep three CTAs per SM if
// the registers allow (<= 72 per thread at 288 threads); the other modes are
// limited to one or two CTAs by shared or tensor memory and keep the
// compiler's own register choice (each instantiation unit compiles one mode).
#if defined(GP_TC_MODE) && GP_TC_MODE == 2
#define GP_TC_BOUNDS __launch_bounds__(kTcThreads, 3)
#else
#define GP_TC_BOUNDS __launch_bounds__(kTcThreads)
#endif
__global__ void GP_TC_BOUNDS
    kmv_tc_kernel(TcArgs a, int n_cols, int64_t nr_pad, int jtiles, int jt_per_split,
                  uint32_t idesc, uint32_t tmem_cols, int nbs) {
  // nbs: stages of the point / B-operand ring, 2 <= nbs <= kTcBStages (host-chosen
  // to fit shared memory).  ATM_T: A in tensor memory (split BF16 only; the host
  // chooses the instantiation per launch).
  using G = TcGeom<MODE>;
  constexpr int DP = DimTraits<DT>::DP;
  constexpr int NSA = TcTraits<MODE>::NSA;
  constexpr int NSB = TcTraits<MODE>::NSB;
  constexpr int NPROD = TcTraits<MODE>::NPROD;
  constexpr int EPC = G::EPC;
  constexpr int NMAT = GRAD ? 2 : 1;
  constexpr int HALF_CK = G::CK / 2;
  constexpr bool ATM = TcATmem<MODE>::ON && ATM_T;   // A operand in tensor memory
  constexpr uint32_t ACOLS = TcATmem<MODE>::COLS;

  if (a.active != nullptr && *a.active == 0) return;

  extern __shared__ __align__(1024) unsigned char smem[];
  const TcSmem L = tc_smem<MODE, DT>(n_cols, GRAD, nbs, ATM);
  uint64_t* fullX = reinterpret_cast<uint64_t*>(smem + L.bars);  // [nbs] points + B landed
  uint64_t* emptyX = fullX + kTcBStages;                          // [nbs] MMA done with stage
  uint64_t* fullA = emptyX + kTcBStages;                          // [2] A written (256 arrivals)
  uint64_t* emptyA = fullA + kTcAStages;                          // [2] MMA done with A
  uint64_t* folded = emptyA + kTcAStages;                         // [1] block sum folded
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(folded + 1);
  int* abort_s = reinterpret_cast<int*>(tmem_holder + 1);
  float* sX = reinterpret_cast<float*>(smem + L.sx);
  unsigned char* sB = smem + L.sb;
  unsigned char* sA = smem + L.sa;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const bool is_eval = warp < 8;
  const int m = tid & (kTcM - 1);        // row within the tile (eval warps)
  const int half = (tid >> 7) & 1;       // which half of the tile's columns
  const int quad = warp & 3;             // tensor-memory lane quadrant
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kTcM + m;
  const int s = blockIdx.y;
  const int jt0 = s * jt_per_split;
  const int jt1 = min(jt0 + jt_per_split, jtiles);
  const int T = jt1 - jt0;
  const int acc_cols = NMAT * n_cols;    // accumulator columns = running-sum columns
  // Tensor-memory column of A matrix (stage, K or D, hi or lo) when ATM.
  auto a_col = [&](int st, int mat, int part) -> uint32_t {
    return static_cast<uint32_t>(2 * acc_cols) +
           static_cast<uint32_t>((st * NMAT + mat) * NSA + part) * ACOLS;
  };

  if (tid == 0) {
    for (int i = 0; i < kTcBStages; ++i) {
      dev::mbar_init(&fullX[i], 1);
      dev::mbar_init(&emptyX[i], 1);
    }
    for (int i = 0; i < kTcAStages; ++i) {
      dev::mbar_init(&fullA[i], kTcEvalThreads);
      dev::mbar_init(&emptyA[i], 1);
    }
    dev::mbar_init(folded, kTcEvalThreads);
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

  auto set_abort = [&]() {
    atomicExch(abort_s, 1);
    atomicExch(a.err, kDevTimeout);
  };

  if (is_eval) {
    // ------------------------------------------------------------ eval warps
    float2 xi2[DT];
    load_row_point<DT>(a.xr, row, xi2);
    {
      // Zero the running sums: warp (quad, half) clears chunks c % 2 == half.
      uint32_t z[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) z[u] = 0u;
      for (int c0 = 16 * half; c0 < acc_cols; c0 += 32)
        tc::st16(tmem + lane_base + static_cast<uint32_t>(acc_cols + c0), z);
      tc::wait_st();
    }
    const uint32_t rowoff =
        static_cast<uint32_t>(m >> 3) * G::SBO + static_cast<uint32_t>(m & 7) * 16;
    bool ok = true;
    int bs = 0;          // ring slot of tile t and the parity of its phase,
    uint32_t bph = 0;    // advanced without division
    for (int t = 0; t < T && ok; ++t, bph ^= (++bs == nbs), bs = bs == nbs ? 0 : bs) {
      const int as = t % kTcAStages;
      ok = tc::wait_or_abort(&fullX[bs], bph, abort_s);
      if (ok && t >= kTcAStages)
        ok = tc::wait_or_abort(&emptyA[as], ((t - kTcAStages) / kTcAStages) & 1, abort_s);
      if (!ok) break;
      if constexpr (ATM) tc::fence_after();   // the MMAs that read this A stage are complete
      const float* xs = sX + bs * (L.xbytes / 4);
      const int jo = ((jt0 + t) * G::BK) & (kTcBK - 1);   // the tile's offset in its point tile
      unsigned char* aK = sA + (as * NMAT * NSA) * L.abytes;
      unsigned char* aD = aK + NSA * L.abytes;
      // ATM: this thread's 16 entries of its row as 8 packed words per matrix.
      uint32_t wK[ATM ? 2 : 1][8], wD[ATM ? 2 : 1][8];
#pragma unroll
      for (int kh = 0; kh < HALF_CK; ++kh) {
        const int kg = half * HALF_CK + kh;
        float2 kv[EPC / 2], dv[EPC / 2];
#pragma unroll
        for (int u = 0; u < EPC / 4; ++u) {
          float2 q01, q23;
          sqdist_quad<DT>(xi2, xs, jo + kg * EPC + 4 * u, q01, q23);
          dv[2 * u] = dv[2 * u + 1] = make_float2(0.f, 0.f);
          eval_pair<KIND, GRAD>(q01, kv[2 * u], dv[2 * u]);
          eval_pair<KIND, GRAD>(q23, kv[2 * u + 1], dv[2 * u + 1]);
        }
        if constexpr (ATM) {
          tc::pack_bf16<true>(kv, &wK[0][4 * kh], &wK[1][4 * kh]);
          if constexpr (GRAD) tc::pack_bf16<true>(dv, &wD[0][4 * kh], &wD[1][4 * kh]);
        } else {
          const uint32_t off = rowoff + static_cast<uint32_t>(kg) * G::LBO;
          tc::store_group<MODE, (NSA == 2)>(aK, aK + L.abytes, off, kv);
          if constexpr (GRAD) tc::store_group<MODE, (NSA == 2)>(aD, aD + L.abytes, off, dv);
        }
      }
      if constexpr (ATM) {
        static_assert(HALF_CK == 2 && NSA == 2, "A in tensor memory: 16 entries, hi and lo");
        const uint32_t lcol = lane_base + static_cast<uint32_t>(half * 8);
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          tc::st8(tmem + lcol + a_col(as, 0, part), wK[part]);
          if constexpr (GRAD) tc::st8(tmem + lcol + a_col(as, 1, part), wD[part]);
        }
        tc::wait_st();
        tc::fence_before();
      } else {
        tc::fence_proxy_async();
      }
      tc::arrive(&fullA[as]);
      if (t > 0 && t % G::FLUSH == 0) {
        // Fold the block that ended at tile t-1 once its MMAs are complete.
        ok = tc::wait_or_abort(&emptyA[(t - 1) % kTcAStages], ((t - 1) / kTcAStages) & 1, abort_s);
        if (!ok) break;
        tc::fence_after();
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
        tc::fence_before();
        tc::arrive(folded);
      }
    }
    if (ok && T > 0)
      ok = tc::wait_or_abort(&emptyA[(T - 1) % kTcAStages], ((T - 1) / kTcAStages) & 1, abort_s);
    if (!ok) {
      set_abort();
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
  } else if (tid == kTcEvalThreads) {
    // ---------------------------------------------------- control warp, lane 0
    int issued = 0;       // tiles whose copies were issued
    int committed = -1;   // last tile whose MMAs were committed
    int ist = 0;         // ring slot of the next copy to issue
    auto issue_copy = [&](int t) {
      const int st = ist;
      ist = (ist + 1 == nbs) ? 0 : ist + 1;
      const int64_t jt = jt0 + t;
      dev::mbar_arrive_expect_tx(&fullX[st], L.xbytes + NSB * L.bbytes);
      dev::bulk_g2s(sX + st * (L.xbytes / 4), a.xc + ((jt * G::BK) / kTcBK) * kTcBK * DP, L.xbytes,
                    &fullX[st]);
      const unsigned char* vsrc = static_cast<const unsigned char*>(a.vt) + jt * NSB * L.bbytes;
      dev::bulk_g2s(sB + st * NSB * L.bbytes, vsrc, NSB * L.bbytes, &fullX[st]);
    };
    // Descriptor templates of stage 0 (addresses < 256 KiB keep the 14-bit
    // start-address field free of carries when offsets are added).
    const uint64_t desc_a0 = tc::smem_desc(dev::smem_addr(sA), G::LBO, G::SBO);
    const uint64_t desc_b0 = tc::smem_desc(dev::smem_addr(sB), G::LBO, G::SBO);
    const uint32_t a_stage = NMAT * NSA * L.abytes;   // bytes per A stage
    const uint32_t b_stage = NSB * L.bbytes;          // bytes per B stage
    // Prefetch distance: nbs - 1 tiles ahead of the tile being consumed.
    const int kAhead = nbs - 1;
    for (int t = 0; t < kAhead && t < T; ++t) issue_copy(t);
    issued = T < kAhead ? T : kAhead;
    bool ok = true;
    int bs = 0, pbs = 0;           // ring slot of tile t, and of tile t-1
    uint32_t bph = 0, pbph = 0;    // their phase parities
    for (int t = 0; t < T; ++t) {
      if (t > 0) {
        pbs = bs;
        pbph = bph;
        if (++bs == nbs) {
          bs = 0;
          bph ^= 1u;
        }
      }
      const int as = t % kTcAStages;
      ok = tc::wait_or_abort(&fullX[bs], bph, abort_s);
      if (ok) ok = tc::wait_or_abort(&fullA[as], (t / kTcAStages) & 1, abort_s);
      if (ok && t > 0 && t % G::FLUSH == 0)
        ok = tc::wait_or_abort(folded, ((t / G::FLUSH) - 1) & 1, abort_s);
      if (!ok) break;
      tc::fence_after();
      // Descriptors: the stage-0 templates plus this tile's offsets, in the
      // descriptor's start-address units (bytes >> 4, the low bits).
      const uint64_t da = desc_a0 + ((static_cast<uint32_t>(as) * a_stage) >> 4);
      const uint64_t db = desc_b0 + ((static_cast<uint32_t>(bs) * b_stage) >> 4);
      uint32_t acc = (t % G::FLUSH == 0) ? 0u : 1u;   // a block starts from zero
#pragma unroll
      for (int ks = 0; ks < G::KSTEPS; ++ks) {
        // One MMA consumes two K-adjacent core matrices (32 bytes of K).
        const uint64_t ko = (static_cast<uint64_t>(ks) * 2 * G::LBO) >> 4;
        // Products (A part, B part): (hi, hi), then (hi, lo), then (lo, hi).
#pragma unroll
        for (int pr = 0; pr < NPROD; ++pr) {
          const uint64_t am = (pr == 2) ? 1u : 0u;
          const uint64_t bm = (pr == 1) ? 1u : 0u;
          const uint64_t bdesc = db + ((bm * L.bbytes) >> 4) + ko;
          if constexpr (ATM) {
            // One MMA takes 16 K values = 8 columns of the A matrix.
            const uint32_t kc = static_cast<uint32_t>(ks * 8);
            tc::mma_ts<MODE>(tmem, tmem + a_col(as, 0, static_cast<int>(am)) + kc, bdesc, idesc, acc);
            if constexpr (GRAD)
              tc::mma_ts<MODE>(tmem + static_cast<uint32_t>(n_cols),
                               tmem + a_col(as, 1, static_cast<int>(am)) + kc, bdesc, idesc, acc);
          } else {
            tc::mma<MODE>(tmem, da + ((am * L.abytes) >> 4) + ko, bdesc, idesc, acc);
            if constexpr (GRAD)
              tc::mma<MODE>(tmem + static_cast<uint32_t>(n_cols),
                            da + (((NSA + am) * L.abytes) >> 4) + ko, bdesc, idesc, acc);
          }
          acc = 1u;
        }
      }
      tc::commit(&emptyA[as]);
      tc::commit(&emptyX[bs]);
      committed = t;
      // Prefetch tile t + kAhead into the stage tile t-1 used, once its MMAs are done.
      if (issued < T) {
        if (t >= 1)
          ok = tc::wait_or_abort(&emptyX[pbs], pbph, abort_s);
        if (!ok) break;
        issue_copy(issued);
        ++issued;
      }
    }
    if (!ok) {
      set_abort();
      // Wait (bounded) for the MMAs and copies this thread put in flight.
      if (committed >= 0)
        dev::mbar_wait(&emptyA[committed % kTcAStages], (committed / kTcAStages) & 1);
      for (int t = committed + 1; t < issued; ++t)
        dev::mbar_wait(&fullX[t % nbs], (t / nbs) & 1);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

}  // namespace gp
