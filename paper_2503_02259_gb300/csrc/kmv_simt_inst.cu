// Instantiations of the SIMT product for one (kernel family, grad, dimension)
// triple.  Compiled once per triple with -DGP_KIND=<0|1> -DGP_GRAD=<0|1>
// -DGP_DT=<1|2|3|4|8|16> so that the instantiations build in parallel
// translation units.
#include <algorithm>
#include <atomic>

#include "kmv_simt.cuh"

#if !defined(GP_KIND) || !defined(GP_GRAD) || !defined(GP_DT)
#error "GP_KIND, GP_GRAD and GP_DT must be defined"
#endif

#define GP_CAT6(a, b, c, d, e, f) a##b##c##d##e##f
#define GP_FN(prefix, k, g, dt) GP_CAT6(prefix, k, _g, g, _d, dt)
#define GP_LAUNCH GP_FN(launch_simt_k, GP_KIND, GP_GRAD, GP_DT)
#define GP_OCC GP_FN(occupancy_simt_k, GP_KIND, GP_GRAD, GP_DT)
#define GP_GLAUNCH GP_FN(launch_simt_group_k, GP_KIND, GP_GRAD, GP_DT)

namespace gp {

namespace {

constexpr size_t kMaxDynSmem = 160 * 1024;

template <int DT, int TW>
auto kernel_ptr() {
  return kmv_simt_kernel<GP_KIND, (GP_GRAD != 0), DT, TW>;
}

// Raise the dynamic shared-memory cap once per device and instantiation.
template <int DT, int TW>
cudaError_t ensure_attr() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel_ptr<DT, TW>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kMaxDynSmem));
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <int DT, int TW>
cudaError_t launch_one(const SimtPlan& p, const SimtArgs& a, cudaStream_t st) {
  cudaError_t e = ensure_attr<DT, TW>();
  if (e != cudaSuccess) return e;
  const size_t smem = simt_smem_bytes(DimTraits<DT>::DP, p.w_pad);
  dim3 grid(p.row_tiles, p.split);
  auto fn = kernel_ptr<DT, TW>();
  fn<<<grid, kThreads, smem, st>>>(a, p.w_pad, p.ng, p.nr_pad, p.jtiles, p.jt_per_split);
  count_launch();
  return cudaGetLastError();
}

template <int DT, int TW>
auto group_ptr() {
  return kmv_simt_group_kernel<GP_KIND, (GP_GRAD != 0), DT, TW>;
}

// The grouped (persistent) product: as many CTAs as fit on the device at once,
// at most one per work item.
template <int DT, int TW>
cudaError_t launch_group_one(const SimtPlan& p, const SimtGroup& g, cudaStream_t st) {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(group_ptr<DT, TW>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kMaxDynSmem));
    if (e != cudaSuccess) return e;
    done.fetch_or(bit, std::memory_order_acq_rel);
  }
  const size_t smem = simt_smem_bytes(DimTraits<DT>::DP, p.w_pad);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, group_ptr<DT, TW>(), kThreads, smem) !=
          cudaSuccess ||
      nb < 1)
    nb = 1;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
  const int blocks = std::max(1, std::min(g.total_items, nb * sms));
  auto fn = group_ptr<DT, TW>();
  fn<<<blocks, kThreads, smem, st>>>(g, p.w_pad, p.ng);
  count_launch();
  return cudaGetLastError();
}

template <int DT, int TW>
int occ_one(int w_pad) {
  if (ensure_attr<DT, TW>() != cudaSuccess) return 1;
  int nb = 0;
  const size_t smem = simt_smem_bytes(DimTraits<DT>::DP, w_pad);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_ptr<DT, TW>(), kThreads, smem) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

#define GP_TW_SWITCH(DT, CALL)                 \
  switch (tw) {                                \
    case 4: return CALL(DT, 4);                \
    case 8: return CALL(DT, 8);                \
    case 12: return CALL(DT, 12);              \
    case 16: return CALL(DT, 16);              \
    case 20: return CALL(DT, 20);              \
    case 24: return CALL(DT, 24);              \
    case 28: return CALL(DT, 28);              \
    case 32: return CALL(DT, 32);              \
    case 36: return CALL(DT, 36);              \
    case 40: return CALL(DT, 40);              \
    default: break;                            \
  }

}  // namespace

cudaError_t GP_LAUNCH(const SimtPlan& p, const SimtArgs& a, cudaStream_t st) {
  const int tw = p.tw;
#define GP_CALL_LAUNCH(D, W) launch_one<D, W>(p, a, st)
  GP_TW_SWITCH(GP_DT, GP_CALL_LAUNCH)
#undef GP_CALL_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t GP_GLAUNCH(const SimtPlan& p, const SimtGroup& g, cudaStream_t st) {
  switch (p.tw) {
    case 4: return launch_group_one<GP_DT, 4>(p, g, st);
    case 12: return launch_group_one<GP_DT, 12>(p, g, st);
    case 20: return launch_group_one<GP_DT, 20>(p, g, st);
    case 36: return launch_group_one<GP_DT, 36>(p, g, st);
    default: return cudaErrorInvalidValue;
  }
}

int GP_OCC(int tw, int w_pad) {
#define GP_CALL_OCC(D, W) occ_one<D, W>(w_pad)
  GP_TW_SWITCH(GP_DT, GP_CALL_OCC)
#undef GP_CALL_OCC
  return 1;
}

}  // namespace gp
