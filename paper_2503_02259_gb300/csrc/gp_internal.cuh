// Internal declarations shared by the libgp translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gp.h"

namespace gp {

// ---------------------------------------------------------------------------
// Tiling constants of the on-the-fly product kernels.
// ---------------------------------------------------------------------------
constexpr int kThreads = 128;   // threads per CTA of the SIMT product kernel
constexpr int kBM = 128;        // row tile (points i) per CTA when ng == 1
constexpr int kBN = 64;         // column tile (points j) per pipeline stage
constexpr int kPad = 128;       // point arrays are padded to a multiple of this
constexpr int kMaxSplit = 64;   // largest j-split of one product

// Device error codes written to the workspace status word.
enum DevErr : int { kDevOk = 0, kDevTimeout = 1, kDevBreakdown = 2, kDevNumeric = 3 };

// Bounded spin limit for mbarrier waits (iterations of try_wait, each of which
// may itself suspend for a hardware-defined interval).
constexpr long long kSpinLimit = 1ll << 22;

// ---------------------------------------------------------------------------
// Kernel-evaluation constants derived from Theta (host side).
// The point coordinates are shifted by a reference point and scaled by `cs`
// once, so that the inner loop works on a scaled squared distance q:
//   Gaussian : q = r^2 log2(e) / (2 l^2);  k = 2^-q;        D' = k q
//   Matern32 : q = 3 r^2 / l^2, a = sqrt(q); k = (1+a) 2^-(a log2 e); D' = a^2 e^-a
// and dk/dl = cD * D'  with cD = 2/(l log2 e) (Gaussian) or 1/l (Matern32).
// With per-dimension length-scales l_t (gp_problem.ls) coordinate t is scaled
// by csd[t], the same formula with l_t, and dk/dl_t = ct[t] E dd_t (see
// grad_ard.cu) with ct[t] the cD formula at l_t.
// ---------------------------------------------------------------------------
struct KernelConsts {
  float cs;                  // coordinate scale (isotropic)
  double cD;                 // derivative scale (isotropic)
  bool ard;                  // per-dimension length-scales
  float csd[GP_MAX_DIM];     // coordinate scale per dimension (all cs when isotropic)
  double ct[GP_MAX_DIM];     // derivative scale per dimension (ARD)
};
KernelConsts kernel_consts(int kernel, double l);
KernelConsts kernel_consts(const gp_problem* prob);

// Padded dimension used for the AoS point layout of a problem of dimension d.
int dim_template(int d);   // 1,2,3,4,8,16: the compile-time dimension
int dim_padded(int dt);    // floats per stored point (2,4,8,16)

// Per-launch plan of the SIMT product.
struct SimtPlan {
  int dt;        // dimension template value
  int dp;        // stored floats per point
  int tw;        // columns per thread
  int ng;        // column groups (w_pad = ng * tw)
  int w_pad;
  int bm;        // rows per CTA = kBM / ng
  int64_t nr_pad, nc_pad;
  int row_tiles; // nr_pad / bm
  int jtiles;    // nc_pad / kBN
  int split;     // S
  int jt_per_split;
};
SimtPlan plan_simt(int64_t nr, int64_t nc, int d, int w, bool grad, int kernel);

// Launch the templated SIMT product (kmv_simt.cuh); returns a CUDA error.
struct SimtArgs {
  const float* xr;   // row points, AoS [nr_pad][dp], scaled
  const float* xc;   // column points, AoS [nc_pad][dp], scaled
  const float* v;    // [nc_pad][w_pad]
  float* part_k;     // [S][nr_pad][w_pad]
  float* part_d;     // [S][nr_pad][w_pad] (grad only)
  const int* active; // optional device flag: if non-NULL and *active == 0 the kernel exits
  int* err;          // device status word
};
cudaError_t launch_simt(const SimtPlan& p, int kernel, bool grad, const SimtArgs& a,
                        cudaStream_t st);

// Several problems' products in one persistent launch (kmv_simt_group_kernel):
// the problems share kernel, grad, dimension template, TW, ng and w_pad; the
// table travels as a kernel parameter.  Work items are numbered problem by
// problem: item0 is the first item of entry k, and an entry's items are
// (row tile, split) in row-tile-fastest order.
constexpr int kMaxGroup = 64;
// TW values the grouped product is built for (a group pads w up to one).
constexpr int kGroupTW[4] = {4, 12, 20, 36};
struct SimtGroupEntry {
  SimtArgs a;
  int64_t nr_pad;
  int row_tiles, split, jtiles, jt_per_split;
  int item0;
};
struct SimtGroup {
  int count;
  int total_items;
  int* counter;   // device word, zero before the launch
  SimtGroupEntry e[kMaxGroup];
};
// plan: the shared dt / tw / ng / w_pad (of any member); blocks: persistent CTAs.
cudaError_t launch_simt_group(const SimtPlan& plan, int kernel, bool grad, const SimtGroup& g,
                              cudaStream_t st);
// Occupancy (resident CTAs per SM) of one instantiation.
int simt_occupancy(int kernel, bool grad, int dt, int tw, int w_pad, int dp);

// Thread-local error message.
void set_error(const std::string& msg);

// Cooperative launches (the fused CG step) are allowed on this host thread
// unless switched off; the request server switches them off in its workers, so
// that grids on concurrent streams never wait for one another's residency.
void set_thread_cooperative(bool allowed);
bool thread_cooperative();

// Measurement hooks: every launcher calls count_launch(); the product launch is
// bracketed by profile_product_begin/end (no-ops unless a window is open).
void count_launch();
void profile_product_begin(cudaStream_t st);
void profile_product_end(cudaStream_t st);

}  // namespace gp

// ---------------------------------------------------------------------------
// Device helpers (inline PTX for the bulk-copy engine and mbarriers).
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace gp {

// Staged point arrays hold tiles of 32 points, dimension-major within a tile:
// coordinate t of point i (dp stored coordinates per point) is at
// ((i / 32) * dp + t) * 32 + i % 32.  A tile of 32 points is contiguous.
__host__ __device__ __forceinline__ int64_t pt_index(int64_t i, int t, int dp) {
  return ((i >> 5) * dp + t) * 32 + (i & 31);
}

namespace dev {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t addr = smem_addr(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One bulk global -> shared copy (TMA engine, non-tensor form), completing
// `bytes` transaction bytes on `bar`.  dst/src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace dev
}  // namespace gp
#endif
