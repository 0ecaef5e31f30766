// gp_kernel_matmul_noalloc: the FP32 on-the-fly product Y = Kh V for callers that
// cannot allocate device memory at the point of the call (a plug-in inside a
// host application that owns the allocator, a loop with a fixed memory budget).
// Its scratch is one file-scope static device array instead of a caller
// workspace.  The paper has no counterpart to this entry point.
#include <math.h>

#include <mutex>
#include <string>

#include "gp_api_internal.h"
#include "kmv_simt.cuh"
#include "vec_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = GP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
// In host code the array's name is only a host-side stand-in, so kernels must
// be given this address, never &g_noalloc_scratch.
gp_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gp::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return GP_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    gp::set_error("gp_kernel_matmul_noalloc: device index out of range");
    return GP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      gp::set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return GP_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Scratch layout: staged points | padded V | partial sums | status word.
struct Layout {
  size_t xs, vp, part, err, bytes;
};

Layout layout_for(const gp::SimtPlan& p) {
  Layout L;
  size_t off = 0;
  L.xs = off;
  off = align256(off + static_cast<size_t>(p.nc_pad) * p.dp * sizeof(float));
  L.vp = off;
  off = align256(off + static_cast<size_t>(p.nc_pad) * p.w_pad * sizeof(float));
  L.part = off;
  off = align256(off + static_cast<size_t>(p.split) * p.nr_pad * p.w_pad * sizeof(float));
  L.err = off;
  L.bytes = off + 256;
  return L;
}

// The same product with `split` j-splits (at most the planner's choice).
gp::SimtPlan with_split(gp::SimtPlan p, int split) {
  p.jt_per_split = (p.jtiles + split - 1) / split;
  p.split = (p.jtiles + p.jt_per_split - 1) / p.jt_per_split;
  return p;
}

gp_status fail(gp_status st, const std::string& msg) {
  gp::set_error(msg);
  return st;
}

}  // namespace

extern "C" gp_status gp_kernel_matmul_noalloc(const gp_problem* prob, const float* V, int32_t w,
                                              float* Y, void* stream) {
  if (prob == nullptr || prob->X == nullptr || V == nullptr || Y == nullptr)
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: NULL pointer argument");
  if (prob->n < 1 || prob->d < 1 || prob->d > GP_MAX_DIM)
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: need n >= 1 and 1 <= d <= 16");
  if (w < 1 || w > GP_MAX_COLS)
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: w must be in [1, 128]");
  if (prob->kernel != GP_KERNEL_GAUSSIAN && prob->kernel != GP_KERNEL_MATERN32)
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: unknown kernel");
  const gp_theta& t = prob->theta;
  if (!(t.s > 0) || !(t.f > 0) || !(t.l > 0) || !isfinite(t.s) || !isfinite(t.f) || !isfinite(t.l))
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: theta: s, f, l must be finite and > 0");
  if (prob->n > (int64_t(1) << 31) - 4096)
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: n too large");

  const int64_t n = prob->n;
  // Fit the scratch: the planner's split first, then fewer splits.
  const gp::SimtPlan p0 = gp::plan_simt(n, n, prob->d, w, false, prob->kernel);
  gp::SimtPlan p = p0;
  Layout L = layout_for(p);
  for (int s = p0.split - 1; L.bytes > kScratchBytes && s >= 1; --s) {
    p = with_split(p0, s);
    L = layout_for(p);
  }
  if (L.bytes > kScratchBytes)
    return fail(GP_ERR_ARG, "gp_kernel_matmul_noalloc: n = " + std::to_string(n) + ", w = " +
                                std::to_string(w) + " needs " + std::to_string(L.bytes) +
                                " bytes of scratch, above the static scratch of " +
                                std::to_string(kScratchBytes) + " bytes");

  void* base = nullptr;
  gp_status st = scratch_address(&base);
  if (st != GP_OK) return st;
  char* b = static_cast<char*>(base);
  float* xs = reinterpret_cast<float*>(b + L.xs);
  float* vp = reinterpret_cast<float*>(b + L.vp);
  float* part = reinterpret_cast<float*>(b + L.part);
  int* err = reinterpret_cast<int*>(b + L.err);

  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const gp::KernelConsts kc = gp::kernel_consts(prob);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), cs);
  if (e == cudaSuccess)
    e = gp::launch_stage_points(prob->X, n, prob->d, prob->d, prob->X, kc.csd, p.dp, p.nc_pad, xs, cs);
  // The array keeps the previous call's contents: the pad columns must be zero.
  if (e == cudaSuccess && w != p.w_pad)
    e = cudaMemsetAsync(vp, 0, sizeof(float) * p.nc_pad * p.w_pad, cs);
  if (e == cudaSuccess) e = gp::launch_pad_block(V, n, w, w, vp, p.nc_pad, p.w_pad, 0, cs);
  if (e == cudaSuccess) {
    gp::SimtArgs a{xs, xs, vp, part, nullptr, nullptr, err};
    e = gp::launch_simt(p, prob->kernel, false, a, cs);
  }
  if (e == cudaSuccess) {
    gp::EpiArgs ep{};
    ep.part_k = part;
    ep.split = p.split;
    ep.nr_pad = p.nr_pad;
    ep.w_pad = p.w_pad;
    ep.v = vp;
    ep.n = n;
    ep.w = w;
    ep.cK = t.f * t.f;
    ep.cV = t.s;
    ep.y = Y;
    ep.ldy = w;
    ep.err = err;
    e = gp::launch_epilogue(ep, cs);
  }
  if (e != cudaSuccess)
    return fail(GP_ERR_CUDA, std::string("gp_kernel_matmul_noalloc: ") + cudaGetErrorString(e));
  return GP_OK;
}
