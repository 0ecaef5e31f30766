// Instantiations of the tensor-core product for one operand mode, compiled once
// per mode with -DGP_TC_MODE=<1|2|3|4> (TF32, BF16, split TF32, split BF16).
#include <algorithm>
#include <atomic>

#include <cuda_bf16.h>

#include "kmv_tc_kernel.cuh"

#ifndef GP_TC_MODE
#error "GP_TC_MODE must be defined"
#endif

#define GP_TC_CAT(a, b) a##b
#define GP_TC_NAME(a, b) GP_TC_CAT(a, b)
#define GP_TC_LAUNCH GP_TC_NAME(launch_tc_mode, GP_TC_MODE)

namespace gp {

namespace {

constexpr int MODE = GP_TC_MODE;
using G = TcGeom<MODE>;

// V [nc_pad][n] (FP32) -> per 32-point tile, NSPLIT B-operand matrices (N x 32,
// K-major core matrices), rounded to the operand type (hi/lo for the split).
__global__ void tc_stage_v_kernel(const float* v, int n, int jtiles, unsigned char* vt) {
  constexpr int EPC = G::EPC;
  constexpr int NS = TcTraits<MODE>::NSB;
  const uint32_t bbytes = static_cast<uint32_t>(n / 8) * G::SBO;
  const int64_t total = static_cast<int64_t>(jtiles) * n * G::CK;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int kg = static_cast<int>(e % G::CK);
    const int c = static_cast<int>((e / G::CK) % n);
    const int64_t jt = e / (static_cast<int64_t>(G::CK) * n);
    float2 vals[EPC / 2];
#pragma unroll
    for (int u = 0; u < EPC / 2; ++u) {
      const int64_t j = jt * G::BK + kg * EPC + 2 * u;
      vals[u] = make_float2(v[j * n + c], v[(j + 1) * n + c]);
    }
    const uint32_t off = static_cast<uint32_t>(c >> 3) * G::SBO + static_cast<uint32_t>(kg) * G::LBO +
                         static_cast<uint32_t>(c & 7) * 16;
    unsigned char* base = vt + jt * NS * bbytes;
    tc::store_group<MODE, (NS == 2)>(base, base + bbytes, off, vals);
  }
}

// The instantiation with A in shared memory (ATM = false) or, for split BF16,
// in tensor memory (ATM = true; other modes map it to the shared-memory one).
template <int KIND, bool GRAD, int DT, bool ATM>
auto kernel_ptr() {
  return kmv_tc_kernel<KIND, GRAD, DT, MODE, ATM && TcATmem<MODE>::ON>;
}

template <int KIND, bool GRAD, int DT, bool ATM>
cudaError_t ensure_attr() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel_ptr<KIND, GRAD, DT, ATM>(),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <int KIND, bool GRAD, int DT>
cudaError_t launch_one(const SimtPlan& p, const TcArgs& a, cudaStream_t st) {
  const int n = p.w_pad;
  if (n > 128 || n < 16 || (n & 15)) return cudaErrorNotSupported;
  cudaError_t e = ensure_attr<KIND, GRAD, DT, false>();
  if (e != cudaSuccess) return e;
  if (TcATmem<MODE>::ON && (e = ensure_attr<KIND, GRAD, DT, true>()) != cudaSuccess) return e;
  // Per form of the A operand (shared memory; for split BF16 also tensor
  // memory) and copy-ring depth (2..kTcBStages stages): the resident CTAs per
  // SM, bounded by the 512 tensor-memory columns.  The choice keeps the most
  // resident CTAs, then A in tensor memory (fewer shared-memory stores), then
  // the deepest ring.  A tile's copies (points and one B slice, a few KB from
  // L2) land within a fraction of the time the eval warps spend on one tile,
  // so two stages suffice to hide them, while one more resident CTA adds eval
  // warps to hide the evaluation's latencies.
  int nbs = 0, best_occ = 0;
  bool atm = false;
  uint32_t cols = 0;
  for (int form = TcATmem<MODE>::ON ? 1 : 0; form >= 0; --form) {
    const bool f_atm = form == 1;
    const auto f_fn = f_atm ? kernel_ptr<KIND, GRAD, DT, true>() : kernel_ptr<KIND, GRAD, DT, false>();
    const uint32_t f_cols = tc_tmem_cols<MODE>(n, GRAD, f_atm);
    if (f_cols > 512) continue;
    const int f_max = static_cast<int>(512 / f_cols);
    for (int b = kTcBStages; b >= 2; --b) {
      const TcSmem Lb = tc_smem<MODE, DT>(n, GRAD, b, f_atm);
      if (Lb.total > 227u * 1024u) continue;
      int occ_b = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, f_fn, kTcThreads, Lb.total);
      if (e != cudaSuccess) return e;
      occ_b = std::min(occ_b, f_max);
      if (occ_b > best_occ) {
        best_occ = occ_b;
        nbs = b;
        atm = f_atm;
        cols = f_cols;
      }
    }
  }
  if (nbs == 0) return cudaErrorNotSupported;
  const int max_ctas = static_cast<int>(512 / cols);
  const auto fn = atm ? kernel_ptr<KIND, GRAD, DT, true>() : kernel_ptr<KIND, GRAD, DT, false>();
  const TcSmem L = tc_smem<MODE, DT>(n, GRAD, nbs, atm);
  // Reserve shared memory so that no more CTAs reside on an SM than its 512
  // tensor-memory columns hold: a CTA beyond them would only wait in
  // tcgen05.alloc.  The bound is set from the SM's 228 KB (1 KB of it reserved
  // per CTA) rather than from the occupancy query, which counted two CTAs
  // where three were placed when the A operand left shared memory.
  size_t smem = L.total;
  {
    const size_t per_sm = 228u * 1024u;
    // (smem + 1 KB) x (max_ctas + 1) > 228 KB.
    const size_t floor_smem = per_sm / static_cast<size_t>(max_ctas + 1) + 1;
    smem = std::max(smem, floor_smem);
    if (smem > 227u * 1024u) smem = 227u * 1024u;
  }
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTcThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorNotSupported;
  // Stage V as the B operand.
  {
    const int64_t total = static_cast<int64_t>(p.jtiles) * n * G::CK;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    tc_stage_v_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(a.v, n, p.jtiles,
                                                                static_cast<unsigned char*>(a.vt));
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // Instruction descriptor: FP32 accumulator, operand formats, K-major A and B,
  // N >> 3 at bit 17, M >> 4 at bit 24.
  const uint32_t fmt = TcTraits<MODE>::FMT;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) |
                         (static_cast<uint32_t>(n >> 3) << 17) |
                         (static_cast<uint32_t>(kTcM >> 4) << 24);
  dim3 grid(p.row_tiles, p.split);
  profile_product_begin(st);
  fn<<<grid, kTcThreads, smem, st>>>(a, n, p.nr_pad, p.jtiles, p.jt_per_split, idesc, cols, nbs);
  profile_product_end(st);
  count_launch();
  return cudaGetLastError();
}

#define GP_TC_DT_SWITCH(K, GR)                          \
  switch (p.dt) {                                       \
    case 1:                                             \
    case 2: return launch_one<K, GR, 2>(p, a, st);      \
    case 3: return launch_one<K, GR, 3>(p, a, st);      \
    case 4: return launch_one<K, GR, 4>(p, a, st);      \
    case 8: return launch_one<K, GR, 8>(p, a, st);      \
    case 16: return launch_one<K, GR, 16>(p, a, st);    \
    default: break;                                     \
  }

}  // namespace

cudaError_t GP_TC_LAUNCH(const SimtPlan& p, int kernel, bool grad, const TcArgs& a, cudaStream_t st) {
  if (kernel == 0) {
    if (grad) {
      GP_TC_DT_SWITCH(0, true)
    } else {
      GP_TC_DT_SWITCH(0, false)
    }
  } else {
    if (grad) {
      GP_TC_DT_SWITCH(1, true)
    } else {
      GP_TC_DT_SWITCH(1, false)
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace gp
