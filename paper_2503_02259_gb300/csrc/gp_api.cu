// C ABI of libgp.so (include/gp.h): argument checks, launch planning,
// workspace carving and the host loop of the block CG.  Every arithmetic step
// of the path runs in the kernels of kmv_simt.cuh / kmv_tc.cu / vec_kernels.cu;
// this file only sequences them.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "gp_api_internal.h"
#include "grad_ard.cuh"
#include "nystrom.cuh"
#include "kmv_tc.cuh"
#include "residual.cuh"
#include "vec_kernels.cuh"

namespace gp {

// Per-(kernel, grad, dimension) instantiation units (kmv_simt_inst.cu).
#define GP_SIMT_DECL(K, G, D)                                                                \
  cudaError_t launch_simt_k##K##_g##G##_d##D(const SimtPlan&, const SimtArgs&, cudaStream_t); \
  cudaError_t launch_simt_group_k##K##_g##G##_d##D(const SimtPlan&, const SimtGroup&,           \
                                                   cudaStream_t);                              \
  int occupancy_simt_k##K##_g##G##_d##D(int, int);
#define GP_SIMT_DECL_DT(K, G) \
  GP_SIMT_DECL(K, G, 1)       \
  GP_SIMT_DECL(K, G, 2)       \
  GP_SIMT_DECL(K, G, 3)       \
  GP_SIMT_DECL(K, G, 4)       \
  GP_SIMT_DECL(K, G, 8)       \
  GP_SIMT_DECL(K, G, 16)
GP_SIMT_DECL_DT(0, 0)
GP_SIMT_DECL_DT(0, 1)
GP_SIMT_DECL_DT(1, 0)
GP_SIMT_DECL_DT(1, 1)

#define GP_SIMT_DT_SWITCH(K, G, CALL) \
  switch (dt) {                       \
    case 1: return CALL(K, G, 1);     \
    case 2: return CALL(K, G, 2);     \
    case 3: return CALL(K, G, 3);     \
    case 4: return CALL(K, G, 4);     \
    case 8: return CALL(K, G, 8);     \
    case 16: return CALL(K, G, 16);   \
    default: break;                   \
  }

static cudaError_t launch_simt_dt(int kernel, bool grad, const SimtPlan& p, const SimtArgs& a,
                                  cudaStream_t st) {
  const int dt = p.dt;
#define GP_L(K, G, D) launch_simt_k##K##_g##G##_d##D(p, a, st)
  if (kernel == 0) {
    if (grad) { GP_SIMT_DT_SWITCH(0, 1, GP_L) } else { GP_SIMT_DT_SWITCH(0, 0, GP_L) }
  } else {
    if (grad) { GP_SIMT_DT_SWITCH(1, 1, GP_L) } else { GP_SIMT_DT_SWITCH(1, 0, GP_L) }
  }
#undef GP_L
  return cudaErrorInvalidValue;
}

static cudaError_t launch_simt_group_dt(int kernel, bool grad, const SimtPlan& p, const SimtGroup& g,
                                        cudaStream_t st) {
  const int dt = p.dt;
#define GP_G(K, G, D) launch_simt_group_k##K##_g##G##_d##D(p, g, st)
  if (kernel == 0) {
    if (grad) { GP_SIMT_DT_SWITCH(0, 1, GP_G) } else { GP_SIMT_DT_SWITCH(0, 0, GP_G) }
  } else {
    if (grad) { GP_SIMT_DT_SWITCH(1, 1, GP_G) } else { GP_SIMT_DT_SWITCH(1, 0, GP_G) }
  }
#undef GP_G
  return cudaErrorInvalidValue;
}

static int occupancy_simt_dt(int kernel, bool grad, int dt, int tw, int w_pad) {
#define GP_O(K, G, D) occupancy_simt_k##K##_g##G##_d##D(tw, w_pad)
  if (kernel == 0) {
    if (grad) { GP_SIMT_DT_SWITCH(0, 1, GP_O) } else { GP_SIMT_DT_SWITCH(0, 0, GP_O) }
  } else {
    if (grad) { GP_SIMT_DT_SWITCH(1, 1, GP_O) } else { GP_SIMT_DT_SWITCH(1, 0, GP_O) }
  }
#undef GP_O
  return 1;
}

namespace {
thread_local std::string t_err;

// Measurement window state (per host thread).
struct ProfileState {
  bool on = false;
  int64_t launches = 0;
  int64_t product_launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t used = 0;
};
thread_local ProfileState t_prof;
constexpr size_t kMaxProfiled = 65536;
// Stream capture in progress on this host thread: launches are recorded into a
// graph, not executed, so they are counted separately and not timed.
thread_local int t_capturing = 0;
thread_local bool t_cooperative = true;
thread_local int64_t t_captured_launches = 0;
std::mutex g_mu;
std::map<std::tuple<int, int, int, int, int, int>, int> g_occ;
std::map<int, int> g_nsm;
}  // namespace

void set_error(const std::string& msg) { t_err = msg; }

void set_thread_cooperative(bool allowed) { t_cooperative = allowed; }
bool thread_cooperative() { return t_cooperative; }

void count_launch() {
  if (t_capturing)
    ++t_captured_launches;
  else
    ++t_prof.launches;
}

void profile_product_begin(cudaStream_t st) {
  if (!t_prof.on || t_capturing) return;
  ++t_prof.product_launches;
  if (t_prof.used >= kMaxProfiled) return;
  if (t_prof.used == t_prof.ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    t_prof.ev.emplace_back(a, b);
  }
  cudaEventRecord(t_prof.ev[t_prof.used].first, st);
}

void profile_product_end(cudaStream_t st) {
  if (!t_prof.on || t_capturing || t_prof.used >= t_prof.ev.size()) return;
  cudaEventRecord(t_prof.ev[t_prof.used].second, st);
  ++t_prof.used;
}
const char* last_error_cstr() { return t_err.c_str(); }

KernelConsts kernel_consts(int kernel, double l) {
  KernelConsts k{};
  const double log2e = 1.4426950408889634;
  if (kernel == GP_KERNEL_GAUSSIAN) {
    k.cs = static_cast<float>(sqrt(log2e / 2.0) / l);
    k.cD = 2.0 / (l * log2e);
  } else {
    k.cs = static_cast<float>(sqrt(3.0) / l);
    k.cD = 1.0 / l;
  }
  k.ard = false;
  for (int t = 0; t < GP_MAX_DIM; ++t) {
    k.csd[t] = k.cs;
    k.ct[t] = k.cD;
  }
  return k;
}

KernelConsts kernel_consts(const gp_problem* prob) {
  KernelConsts k = kernel_consts(prob->kernel, prob->theta.l);
  if (prob->ls == nullptr) return k;
  k.ard = true;
  for (int t = 0; t < prob->d && t < GP_MAX_DIM; ++t) {
    const KernelConsts kt = kernel_consts(prob->kernel, prob->ls[t]);
    k.csd[t] = kt.cs;
    k.ct[t] = kt.cD;
  }
  return k;
}

int dim_template(int d) {
  if (d <= 4) return d;
  if (d <= 8) return 8;
  return 16;
}

int dim_padded(int dt) { return dt <= 2 ? 2 : ((dt + 3) / 4) * 4; }

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_nsm.find(dev);
  if (it != g_nsm.end()) return it->second;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    nsm = 152;
  g_nsm[dev] = nsm;
  return nsm;
}

int simt_occupancy(int kernel, bool grad, int dt, int tw, int w_pad, int) {
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, kernel, grad ? 1 : 0, dt, tw, w_pad);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
  }
  int occ = 1;
  occ = occupancy_simt_dt(kernel, grad, dt, tw, w_pad);
  std::lock_guard<std::mutex> lk(g_mu);
  g_occ[key] = occ;
  return occ;
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

SimtPlan plan_simt(int64_t nr, int64_t nc, int d, int w, bool grad, int kernel) {
  SimtPlan p;
  p.dt = dim_template(d);
  p.dp = dim_padded(p.dt);
  // One column group up to 40 columns (a 1 + 32-probe block stays in one group,
  // so each entry is evaluated once), else two or four groups of <= 32.
  p.ng = w <= 40 ? 1 : (w <= 64 ? 2 : 4);
  const int per = (w + p.ng - 1) / p.ng;
  p.tw = static_cast<int>(round_up(per, 4));
  p.w_pad = p.ng * p.tw;
  p.bm = kBM / p.ng;
  p.nr_pad = round_up(nr, kPad);
  p.nc_pad = round_up(nc, kPad);
  p.row_tiles = static_cast<int>(p.nr_pad / p.bm);
  p.jtiles = static_cast<int>(p.nc_pad / kBN);
  // Split the j range so that the CTAs spread evenly over the SMs: minimise
  // (most CTAs on one SM) x (tiles per CTA + fixed cost), lightly penalising
  // the extra partial-sum traffic of each split.
  const int nsm = num_sms();
  int best_s = 1;
  double best = 1e300;
  const int smax = std::min(p.jtiles, kMaxSplit);
  for (int s = 1; s <= smax; ++s) {
    const int jps = (p.jtiles + s - 1) / s;
    const int s_eff = (p.jtiles + jps - 1) / jps;
    if (s_eff != s) continue;
    const int64_t units = static_cast<int64_t>(p.row_tiles) * s_eff;
    const double per_sm = static_cast<double>((units + nsm - 1) / nsm);
    const double cost = per_sm * (jps + 0.5) * (1.0 + 0.002 * s);
    if (cost < best) {
      best = cost;
      best_s = s;
    }
  }
  p.jt_per_split = (p.jtiles + best_s - 1) / best_s;
  p.split = (p.jtiles + p.jt_per_split - 1) / p.jt_per_split;
  (void)grad;
  (void)kernel;
  return p;
}

SimtPlan plan_for(int64_t nr, int64_t nc, int d, int w, bool grad, int kernel, int prec) {
  if (prec == GP_PREC_FP32) return plan_simt(nr, nc, d, w, grad, kernel);
  return plan_tc(nr, nc, d, w, kernel, prec);
}

cudaError_t launch_simt(const SimtPlan& p, int kernel, bool grad, const SimtArgs& a,
                        cudaStream_t st) {
  return launch_simt_dt(kernel, grad, p, a, st);
}

cudaError_t launch_simt_group(const SimtPlan& plan, int kernel, bool grad, const SimtGroup& g,
                              cudaStream_t st) {
  return launch_simt_group_dt(kernel, grad, plan, g, st);
}

// ---------------------------------------------------------------------------
// Workspace carving: a bump allocator over the caller's buffer (256-B aligned).
// ---------------------------------------------------------------------------
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Layout of the product workspace (matmul / grad matmul / predict).
struct ProdWs {
  float* xr;      // row points (== xc for a square product)
  float* xc;
  float* vp;
  float* part_k;
  float* part_d;
  void* vt;       // tensor-core B-operand tiles (NULL for FP32)
  int* err;
  size_t bytes;
};

static ProdWs carve_product(void* ws, const SimtPlan& p, bool grad, bool rect, int prec) {
  Carve c(ws);
  ProdWs w;
  w.xc = c.take<float>(static_cast<size_t>(p.nc_pad) * p.dp);
  w.xr = rect ? c.take<float>(static_cast<size_t>(p.nr_pad) * p.dp) : w.xc;
  w.vp = c.take<float>(static_cast<size_t>(p.nc_pad) * p.w_pad);
  w.part_k = c.take<float>(static_cast<size_t>(p.split) * p.nr_pad * p.w_pad);
  w.part_d = grad ? c.take<float>(static_cast<size_t>(p.split) * p.nr_pad * p.w_pad) : nullptr;
  const size_t vtb = tc_vt_bytes(p, prec);
  w.vt = vtb ? static_cast<void*>(c.take<unsigned char>(vtb)) : nullptr;
  w.err = c.take<int>(64);
  w.bytes = c.off + 256;
  return w;
}

// The CG product (pc, possibly tensor-core) and the FP32 derivative product (pg)
// share the solver arrays: give both the wider padded width.
static void unify_width(SimtPlan& pc, SimtPlan& pg) {
  const int w = std::max(pc.w_pad, pg.w_pad);
  pc.w_pad = w;
  pg.w_pad = w;
}

// Layout of the solver workspace (pcg / slq / loss).
struct SolveWs {
  float* xs;
  float* B;
  float* X;
  float* R;
  float* P;
  float* Q;
  float* part;     // max(split_cg, 2 * split_grad) planes
  float* Lq;       // Lanczos basis: lz_k planes (NULL when no SLQ)
  void* vt;        // tensor-core B-operand tiles (NULL for FP32)
  double* red;
  CgState* S;      // block-CG state
  CgState* S2;     // Lanczos state
  size_t bytes;
};

static SolveWs carve_solve(void* ws, const SimtPlan& pc, const SimtPlan& pg, const SimtPlan& pl,
                           bool with_grad, int lz_k, int prec, int slq_prec) {
  Carve c(ws);
  SolveWs w;
  const size_t plane = static_cast<size_t>(pc.nr_pad) * pc.w_pad;
  w.xs = c.take<float>(static_cast<size_t>(pc.nc_pad) * pc.dp);
  w.B = c.take<float>(plane);
  w.X = c.take<float>(plane);
  w.R = c.take<float>(plane);
  w.P = c.take<float>(plane);
  w.Q = c.take<float>(plane);
  size_t planes = std::max<size_t>(pc.split, with_grad ? 2 * static_cast<size_t>(pg.split) : 0);
  if (lz_k > 0) planes = std::max<size_t>(planes, pl.split);
  w.part = c.take<float>(planes * plane);
  w.Lq = lz_k > 0 ? c.take<float>(static_cast<size_t>(lz_k) * plane) : nullptr;
  size_t vtb = tc_vt_bytes(pc, prec);
  if (lz_k > 0) vtb = std::max(vtb, tc_vt_bytes(pl, slq_prec));
  w.vt = vtb ? static_cast<void*>(c.take<unsigned char>(vtb)) : nullptr;
  w.red = c.take<double>(red_doubles(pc.nr_pad, pc.w_pad));
  w.S = c.take<CgState>(1);
  w.S2 = c.take<CgState>(1);
  w.bytes = c.off + 256;
  return w;
}

// Plans of one solver call: the CG product (pc, arithmetic prec), the FP32
// derivative product of the gradient pass (pg) and the SLQ Lanczos product
// (pl, arithmetic slq_prec); they share the solver arrays, so all take the
// widest padded width.
struct SolvePlans {
  SimtPlan pc, pg, pl;
};

static SolvePlans solve_plans(const gp_problem* prob, int w, int prec, int lz_k, int slq_prec) {
  const int64_t n = prob->n;
  SolvePlans P;
  P.pc = plan_for(n, n, prob->d, w, false, prob->kernel, prec);
  P.pg = plan_for(n, n, prob->d, w, true, prob->kernel, GP_PREC_FP32);
  P.pl = lz_k > 0 ? plan_for(n, n, prob->d, w, false, prob->kernel, slq_prec) : P.pc;
  unify_width(P.pc, P.pg);
  unify_width(P.pc, P.pl);
  unify_width(P.pg, P.pl);
  return P;
}

}  // namespace gp

using namespace gp;

// ---------------------------------------------------------------------------
// Argument checks.
// ---------------------------------------------------------------------------
static gp_status fail(gp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

static gp_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GP_CUDA(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static gp_status check_problem(const gp_problem* prob) {
  if (prob == nullptr) return fail(GP_ERR_ARG, "problem is NULL");
  if (prob->X == nullptr) return fail(GP_ERR_ARG, "problem->X is NULL");
  if (prob->n < 1) return fail(GP_ERR_ARG, "n must be >= 1");
  if (prob->d < 1 || prob->d > GP_MAX_DIM) return fail(GP_ERR_ARG, "d must be in [1, 16]");
  if (prob->kernel != GP_KERNEL_GAUSSIAN && prob->kernel != GP_KERNEL_MATERN32)
    return fail(GP_ERR_ARG, "unknown kernel");
  const gp_theta& t = prob->theta;
  if (!(t.s > 0) || !(t.f > 0) || !(t.l > 0) || !isfinite(t.s) || !isfinite(t.f) || !isfinite(t.l))
    return fail(GP_ERR_ARG, "theta: s, f, l must be finite and > 0");
  if (prob->n > (int64_t(1) << 31) - 4096) return fail(GP_ERR_ARG, "n too large");
  if (prob->ls != nullptr)
    for (int t = 0; t < prob->d; ++t)
      if (!(prob->ls[t] > 0) || !isfinite(prob->ls[t]))
        return fail(GP_ERR_ARG, "ls: every per-dimension length-scale must be finite and > 0");
  return GP_OK;
}

static gp_status no_ard(const gp_problem* prob, const char* what) {
  if (prob->ls != nullptr)
    return fail(GP_ERR_UNIMPLEMENTED,
                std::string(what) + " takes an isotropic length-scale (problem->ls must be NULL)");
  return GP_OK;
}

static gp_status check_width(int32_t w) {
  if (w < 1 || w > GP_MAX_COLS) return fail(GP_ERR_ARG, "w must be in [1, 128]");
  return GP_OK;
}

static gp_status check_opts(const gp_solve_opts* o, bool need_probes, bool precond_ok = false) {
  if (o == nullptr) return fail(GP_ERR_ARG, "opts is NULL");
  if (o->precond_rank < 0 || o->precond_rank > GP_MAX_PRECOND_RANK)
    return fail(GP_ERR_ARG, "precond_rank must be in [0, 4096]");
  if (o->precond_rank > 0 && !precond_ok)
    return fail(GP_ERR_UNIMPLEMENTED,
                "the Nystrom preconditioner is taken by gp_pcg_solve and gp_pcg_solve_refined only");
  if (!(o->precond_tol <= 1.0) && !(o->precond_tol > 1.0))
    return fail(GP_ERR_ARG, "precond_tol is NaN");
  if (o->nprobe < 0 || o->nprobe + 1 > GP_MAX_COLS) return fail(GP_ERR_ARG, "nprobe must be in [0, 127]");
  if (need_probes && o->nprobe < 1) return fail(GP_ERR_ARG, "nprobe must be >= 1");
  if (o->nlanczos < 1 || o->nlanczos > GP_MAX_LANCZOS)
    return fail(GP_ERR_ARG, "nlanczos must be in [1, 64]");
  if (!(o->cg_rtol >= 0)) return fail(GP_ERR_ARG, "cg_rtol must be >= 0");
  if (o->prec < GP_PREC_FP32 || o->prec > GP_PREC_BF16X3) return fail(GP_ERR_ARG, "unknown precision");
  if (o->slq_prec != GP_PREC_SAME && (o->slq_prec < GP_PREC_FP32 || o->slq_prec > GP_PREC_BF16X3))
    return fail(GP_ERR_ARG, "unknown slq_prec");
  return GP_OK;
}

static gp_status check_prec(int32_t prec) {
  if (prec < GP_PREC_FP32 || prec > GP_PREC_BF16X3) return fail(GP_ERR_ARG, "unknown precision");
  return GP_OK;
}

static gp_status check_ws(void* ws, size_t have, size_t need) {
  if (ws == nullptr) return fail(GP_ERR_ARG, "workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0)
    return fail(GP_ERR_ARG, "workspace must be 256-byte aligned");
  if (have < need)
    return fail(GP_ERR_OOM, "workspace too small: need " + std::to_string(need) + " bytes, have " +
                                std::to_string(have));
  return GP_OK;
}

static gp_status device_status(const int* err_dev, cudaStream_t st) {
  int h = 0;
  GP_CUDA(cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  if (h == kDevTimeout) return fail(GP_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h == kDevBreakdown) return fail(GP_ERR_BREAKDOWN, "CG breakdown (p^T Kh p <= 0 or non-finite)");
  if (h == kDevNumeric) return fail(GP_ERR_NUMERIC, "non-positive Lanczos eigenvalue");
  return GP_OK;
}

// ---------------------------------------------------------------------------
// Products.
// ---------------------------------------------------------------------------
namespace gp {

// One fused product Kh-sums of V into part_k / part_d (square, points staged).
gp_status run_product(const SimtPlan& p, int kernel, bool grad, int prec, const float* xr,
                      const float* xc, const float* vp, void* vt, float* part_k, float* part_d,
                      const int* active, int* err, cudaStream_t st) {
  if (prec != GP_PREC_FP32) {
    TcArgs ta{xr, xc, vp, vt, part_k, part_d, active, err};
    cudaError_t e = launch_tc(p, kernel, grad, prec, ta, st);
    if (e == cudaErrorNotSupported)
      return fail(GP_ERR_UNIMPLEMENTED, "tensor-core path not available for this shape");
    if (e != cudaSuccess) return cuda_fail(e, "launch_tc");
    return GP_OK;
  }
  SimtArgs a{xr, xc, vp, part_k, part_d, active, err};
  profile_product_begin(st);
  cudaError_t e = launch_simt(p, kernel, grad, a, st);
  profile_product_end(st);
  if (e != cudaSuccess) return cuda_fail(e, "launch_simt");
  return GP_OK;
}

}  // namespace gp

static gp_status product_call(const gp_problem* prob, const float* V, int32_t w, float* Y,
                              float* dYf, float* dYl, bool grad, int32_t prec, void* ws,
                              size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_width(w)) != GP_OK) return s;
  if ((s = check_prec(prec)) != GP_OK) return s;
  if (V == nullptr || Y == nullptr) return fail(GP_ERR_ARG, "V and Y must be non-NULL");
  if (grad && dYl != nullptr && (s = no_ard(prob, "the dKh/dl product")) != GP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = prob->n;
  const SimtPlan p = plan_for(n, n, prob->d, w, grad, prob->kernel, prec);
  ProdWs L = carve_product(nullptr, p, grad, false, prec);
  if ((s = check_ws(ws, ws_bytes, L.bytes)) != GP_OK) return s;
  L = carve_product(ws, p, grad, false, prec);
  const KernelConsts kc = kernel_consts(prob);
  GP_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int), st));
  GP_CUDA(launch_stage_points(prob->X, n, prob->d, prob->d, prob->X, kc.csd, p.dp, p.nc_pad, L.xc, st));
  if (w != p.w_pad) GP_CUDA(cudaMemsetAsync(L.vp, 0, sizeof(float) * p.nc_pad * p.w_pad, st));
  GP_CUDA(launch_pad_block(V, n, w, w, L.vp, p.nc_pad, p.w_pad, 0, st));
  if ((s = run_product(p, prob->kernel, grad, prec, L.xc, L.xc, L.vp, L.vt, L.part_k, L.part_d,
                       nullptr, L.err, st)) != GP_OK)
    return s;
  const double f = prob->theta.f;
  EpiArgs e{};
  e.part_k = L.part_k;
  e.part_d = L.part_d;
  e.split = p.split;
  e.nr_pad = p.nr_pad;
  e.w_pad = p.w_pad;
  e.v = L.vp;
  e.n = n;
  e.w = w;
  e.cK = f * f;
  e.cV = prob->theta.s;
  e.cF = 2.0 * f;
  e.cL = f * f * kc.cD;
  e.y = Y;
  e.ldy = w;
  e.dyf = grad ? dYf : nullptr;
  e.ldf = w;
  e.dyl = grad ? dYl : nullptr;
  e.ldl = w;
  e.err = L.err;
  GP_CUDA(launch_epilogue(e, st));
  return GP_OK;
}

// ---------------------------------------------------------------------------
// Nystrom preconditioner of a solve (nystrom.cuh): the preconditioned residual
// plane Z and the factor's workspace, placed after the solver's workspace.
// ---------------------------------------------------------------------------
namespace gp {

struct Precond {
  NysWs ws;
  float* Z = nullptr;   // [n_pad][w_pad]: z = M^-1 r in PCG; M^-1 of the probe block in the loss
  float* U = nullptr;   // [n_pad][w_pad]: preconditioned Lanczos work vector (loss only)
  float* Lp = nullptr;  // lz_k planes [n_pad][w_pad]: M-images of the Lanczos basis (loss only)
  int rank = 0;
  double s = 0.0;
};

static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// The preconditioner's planes, then its factor workspace.  lz_k > 0 adds the
// Lanczos work plane and lz_k M-image planes; deriv adds dL/dl (the loss).
static size_t precond_bytes(int64_t n_pad, int d, int kmax, int w_pad, int lz_k = 0,
                            bool deriv = false) {
  const size_t plane = align256(sizeof(float) * static_cast<size_t>(n_pad) * w_pad);
  const size_t planes = 1 + (lz_k > 0 ? 1 + static_cast<size_t>(lz_k) : 0);
  return planes * plane + nys_bytes(n_pad, d, kmax, w_pad, deriv) + 256;
}

static Precond carve_precond(void* base, int64_t n_pad, int d, int kmax, int w_pad, int lz_k = 0,
                             bool deriv = false) {
  Precond pc;
  char* b = static_cast<char*>(base);
  const size_t plane = align256(sizeof(float) * static_cast<size_t>(n_pad) * w_pad);
  pc.Z = reinterpret_cast<float*>(b);
  size_t off = plane;
  if (lz_k > 0) {
    pc.U = reinterpret_cast<float*>(b + off);
    pc.Lp = reinterpret_cast<float*>(b + off + plane);
    off += (1 + static_cast<size_t>(lz_k)) * plane;
  }
  pc.ws = carve_nys(b + off, n_pad, d, kmax, w_pad, deriv);
  return pc;
}

// The preconditioner computes only the solve's own w columns (rounded up to 4)
// of planes padded wider for a tensor-core product.
static void set_live_width(Precond& pc, int w) {
  pc.ws.w_live = static_cast<int>(std::min<int64_t>(pc.ws.w_pad, round_up(w, 4)));
}

static int precond_kmax(const gp_problem* prob, int rank) {
  return static_cast<int>(std::min<int64_t>(rank, prob->n));
}

}  // namespace gp

// Bytes of the plain (unrefined) solver workspace of gp_pcg_solve.
static size_t solve_bytes(const gp_problem* prob, int w, int prec) {
  SimtPlan pc = plan_for(prob->n, prob->n, prob->d, w, false, prob->kernel, prec);
  SimtPlan pg = plan_for(prob->n, prob->n, prob->d, w, true, prob->kernel, GP_PREC_FP32);
  unify_width(pc, pg);
  return carve_solve(nullptr, pc, pc, pc, false, 0, prec, prec).bytes;
}

// gp_nystrom_apply: the padded V block, then the preconditioner (whose Z plane
// receives M^-1 V).
static size_t nystrom_entry_bytes(const gp_problem* prob, int w, int kmax) {
  const int64_t n_pad = round_up(prob->n, kPad);
  const int w_pad = static_cast<int>(round_up(w, 4));
  return align256(sizeof(float) * static_cast<size_t>(n_pad) * w_pad) +
         precond_bytes(n_pad, prob->d, kmax, w_pad);
}

static gp_status build_precond(const gp_problem* prob, int kmax, double tol, Precond& pc,
                               cudaStream_t st) {
  NysProblem P{prob->X, prob->n, prob->d, prob->kernel, prob->theta.f, prob->theta.l, prob->theta.s,
               prob->ls};
  int rank = 0, derr = 0;
  const double tol_abs = tol > 0 ? tol * prob->theta.f * prob->theta.f : 0.0;
  const cudaError_t e = nys_build(pc.ws, P, kmax, tol_abs, &rank, &derr, st);
  if (e == cudaErrorInvalidValue && derr != 0)
    return fail(GP_ERR_NUMERIC, "Nystrom preconditioner: C = s I + L^T L met a non-positive pivot");
  if (e != cudaSuccess) return cuda_fail(e, "nys_build");
  pc.rank = rank;
  pc.s = prob->theta.s;
  return GP_OK;
}

// ---------------------------------------------------------------------------
// Block CG host loop.
// ---------------------------------------------------------------------------
namespace gp {

// One block-CG iteration: the product K P, then alpha, the x / r update and the
// p update (vec_kernels.cu), as one cooperative launch when `fused`, else as
// three launches with the same arithmetic.
static gp_status cg_iteration(const gp_problem* prob, const SimtPlan& p, int prec, SolveWs& W,
                              bool fused, const Precond* pc, cudaStream_t st) {
  const int64_t n = prob->n;
  const double f2 = prob->theta.f * prob->theta.f;
  gp_status s = run_product(p, prob->kernel, false, prec, W.xs, W.xs, W.P, W.vt, W.part, nullptr,
                            &W.S->n_active, &W.S->err, st);
  if (s != GP_OK) return s;
  if (pc != nullptr) {
    // Preconditioned: alpha = r^T z / p^T Kh p; x, r; z = M^-1 r; beta; p = z + beta p.
    GP_CUDA(launch_cg_epi_alpha(W.S, W.part, p.split, W.P, W.Q, p.nr_pad, n, p.w_pad, f2,
                                prob->theta.s, W.red, st));
    GP_CUDA(launch_pcg_update(W.S, W.X, W.R, W.P, W.Q, p.nr_pad, p.w_pad, W.red, st));
    GP_CUDA(nys_apply(pc->ws, pc->rank, n, pc->s, W.R, pc->Z, &W.S->n_active, st));
    GP_CUDA(launch_pcg_rz(W.S, W.R, pc->Z, p.nr_pad, p.w_pad, false, W.red, st));
    GP_CUDA(launch_cg_pupdate(W.S, pc->Z, W.P, p.nr_pad, p.w_pad, st));
    return GP_OK;
  }
  if (fused) {
    GP_CUDA(launch_cg_step(W.S, W.part, p.split, W.X, W.R, W.P, W.Q, p.nr_pad, n, p.w_pad, f2,
                           prob->theta.s, W.red, st));
    return GP_OK;
  }
  GP_CUDA(launch_cg_epi_alpha(W.S, W.part, p.split, W.P, W.Q, p.nr_pad, n, p.w_pad, f2,
                              prob->theta.s, W.red, st));
  GP_CUDA(launch_cg_update(W.S, W.X, W.R, W.P, W.Q, p.nr_pad, p.w_pad, W.red, st));
  GP_CUDA(launch_cg_pupdate(W.S, W.R, W.P, p.nr_pad, p.w_pad, st));
  return GP_OK;
}

// The fused CG step is used unless the environment sets GP_CG_FUSED=0 (the
// separate kernels give the same bits; the switch exists to compare them).
static bool cg_fused_wanted() {
  const char* v = std::getenv("GP_CG_FUSED");
  return v == nullptr || std::strcmp(v, "0") != 0;
}

// A private non-blocking stream of this host thread on the current device,
// used only to capture graphs (the caller's stream may be the legacy default
// stream, which cannot be captured).  Lives as long as the thread.
static cudaStream_t capture_stream() {
  thread_local std::map<int, cudaStream_t> streams;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  streams[dev] = cs;
  return cs;
}

// The launches of one solver iteration captured once as a CUDA graph and then
// replayed on the caller's stream: one graph launch instead of one launch per
// kernel (the small-n iterations are launch-bound).
class IterationGraph {
 public:
  IterationGraph() = default;
  IterationGraph(const IterationGraph&) = delete;
  IterationGraph& operator=(const IterationGraph&) = delete;
  ~IterationGraph() {
    if (exec_ != nullptr) cudaGraphExecDestroy(exec_);
  }
  // Records body(stream) into the graph; false (and no graph) if anything fails.
  template <class Body>
  bool capture(Body&& body) {
    cudaStream_t cs = capture_stream();
    if (cs == nullptr || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ++t_capturing;
    t_captured_launches = 0;
    const gp_status s = body(cs);
    --t_capturing;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    bool ok = s == GP_OK && e == cudaSuccess && g != nullptr &&
              cudaGraphInstantiate(&exec_, g, 0) == cudaSuccess;
    if (g != nullptr) cudaGraphDestroy(g);
    if (!ok) {
      exec_ = nullptr;
      cudaGetLastError();
      return false;
    }
    kernels_ = t_captured_launches;
    return true;
  }
  cudaError_t launch(cudaStream_t st) {
    for (int64_t k = 0; k < kernels_; ++k) count_launch();
    return cudaGraphLaunch(exec_, st);
  }

 private:
  cudaGraphExec_t exec_ = nullptr;
  int64_t kernels_ = 0;
};

gp_status run_cg(const gp_problem* prob, const SimtPlan& p, int prec, SolveWs& W, int w, int maxit,
                 double rtol, cudaStream_t st, const Precond* pc = nullptr) {
  GP_CUDA(launch_cg_init(W.S, W.B, W.X, W.R, W.P, p.nr_pad, p.w_pad, w, maxit, rtol, W.red, st));
  if (pc != nullptr) {
    // z_0 = M^-1 r_0, r^T z, p_0 = z_0.
    GP_CUDA(nys_apply(pc->ws, pc->rank, prob->n, pc->s, W.R, pc->Z, &W.S->n_active, st));
    GP_CUDA(launch_pcg_rz(W.S, W.R, pc->Z, p.nr_pad, p.w_pad, true, W.red, st));
    GP_CUDA(launch_cg_pupdate(W.S, pc->Z, W.P, p.nr_pad, p.w_pad, st));
  }
  int chunk = 4;
  int issued = 0;
  struct {
    int n_active;
    int err;
  } h{1, 0};
  // The first iteration runs eagerly (it also performs the one-time kernel
  // set-up); the rest replay a graph of one iteration, or run eagerly if the
  // graph could not be built.
  IterationGraph graph;
  bool tried = false, use_graph = false;
  const bool fused =
      pc == nullptr && thread_cooperative() && cg_fused_wanted() && cg_step_fits(p.nr_pad);
  while (issued < maxit) {
    const int todo = std::min(chunk, maxit - issued);
    for (int k = 0; k < todo; ++k) {
      if (issued + k > 0 && !tried) {
        tried = true;
        use_graph = graph.capture(
            [&](cudaStream_t cs) { return cg_iteration(prob, p, prec, W, fused, pc, cs); });
      }
      if (use_graph) {
        GP_CUDA(graph.launch(st));
      } else {
        gp_status s = cg_iteration(prob, p, prec, W, fused, pc, st);
        if (s != GP_OK) return s;
      }
    }
    issued += todo;
    GP_CUDA(cudaMemcpyAsync(&h, W.S, sizeof(h), cudaMemcpyDeviceToHost, st));
    GP_CUDA(cudaStreamSynchronize(st));
    if (h.n_active == 0 || h.err != 0) break;
    if (chunk < 32) chunk *= 2;
  }
  if (h.err == kDevTimeout) return fail(GP_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h.err == kDevBreakdown) return fail(GP_ERR_BREAKDOWN, "CG breakdown (p^T Kh p <= 0 or non-finite)");
  return GP_OK;
}

// k Lanczos steps with full reorthogonalisation on columns [col0, col0 + p) of
// W.B, one process per column, then the Gauss quadrature of log (SLQ) into
// W.S2->out[0..1].  Uses W.R as the work vector and W.Lq as the basis.
gp_status run_lanczos(const gp_problem* prob, const SimtPlan& p, int prec, SolveWs& W, int col0,
                      int np, int k, cudaStream_t st) {
  const int64_t n = prob->n;
  const double f2 = prob->theta.f * prob->theta.f;
  const int64_t plane = p.nr_pad * p.w_pad;
  CgState* S = W.S2;
  GP_CUDA(cudaMemsetAsync(S, 0, sizeof(CgState), st));
  GP_CUDA(launch_lz_init(S, W.B, W.Lq, p.nr_pad, p.w_pad, col0, np, W.red, st));
  for (int j = 0; j < k; ++j) {
    const float* Qj = W.Lq + j * plane;
    gp_status s = run_product(p, prob->kernel, false, prec, W.xs, W.xs, Qj, W.vt, W.part, nullptr,
                              &S->n_active, &S->err, st);
    if (s != GP_OK) return s;
    GP_CUDA(launch_lz_epi_alpha(S, W.part, p.split, Qj, W.R, p.nr_pad, n, p.w_pad, f2,
                                prob->theta.s, j, W.red, st));
    GP_CUDA(launch_lz_three_term(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, st));
    GP_CUDA(launch_lz_reorth(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, W.red, st));
    GP_CUDA(launch_lz_reorth(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, W.red, st));
    GP_CUDA(launch_lz_norm_next(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, k, W.red, st));
  }
  GP_CUDA(launch_slq(S, col0, np, k, st));
  return GP_OK;
}

// SLQ on M^-1/2 Kh M^-1/2 (Eq. 1's second term) for columns [col0, col0 + p)
// of the probe block W.B, with pc.Z = M^-1 W.B: Lanczos in the variables
// q = M^-1/2 qh with the M-images P = M Q kept beside the basis (pc.Lp):
// W = Kh q_j, alpha_j = q_j^T W, u = M^-1 W - alpha_j q_j - beta q_{j-1}, M u
// formed explicitly (s u + L L^T u), two reorthogonalisation passes in the
// M-inner product (h = P^T u), beta_j = sqrt(u^T M u).  (Carrying M u by the
// three-term recurrence instead would divide its error by beta_j at every
// step: with M close to Kh, beta_j is ~1e-4 and the images drift within a
// few steps.)  The quadrature weight is ||zh||^2 = z^T M^-1 z.
gp_status run_lanczos_m(const gp_problem* prob, const SimtPlan& p, int prec, SolveWs& W,
                        const Precond& pc, int col0, int np, int k, cudaStream_t st) {
  const int64_t n = prob->n;
  const double f2 = prob->theta.f * prob->theta.f;
  const int64_t plane = p.nr_pad * p.w_pad;
  CgState* S = W.S2;
  GP_CUDA(cudaMemsetAsync(S, 0, sizeof(CgState), st));
  GP_CUDA(launch_lz_init_m(S, W.B, pc.Z, W.Lq, pc.Lp, p.nr_pad, p.w_pad, col0, np, W.red, st));
  for (int j = 0; j < k; ++j) {
    const float* Qj = W.Lq + j * plane;
    gp_status s = run_product(p, prob->kernel, false, prec, W.xs, W.xs, Qj, W.vt, W.part, nullptr,
                              &S->n_active, &S->err, st);
    if (s != GP_OK) return s;
    GP_CUDA(launch_lz_epi_alpha(S, W.part, p.split, Qj, W.R, p.nr_pad, n, p.w_pad, f2,
                                prob->theta.s, j, W.red, st));
    GP_CUDA(nys_apply(pc.ws, pc.rank, n, pc.s, W.R, pc.U, &S->n_active, st));
    GP_CUDA(launch_lz_three_term(S, pc.U, W.Lq, p.nr_pad, p.w_pad, j, st));
    GP_CUDA(nys_apply_m(pc.ws, pc.rank, n, pc.s, pc.U, W.R, &S->n_active, st));
    GP_CUDA(launch_lz_reorth_m(S, pc.U, W.R, W.Lq, pc.Lp, p.nr_pad, p.w_pad, j, W.red, st));
    GP_CUDA(launch_lz_reorth_m(S, pc.U, W.R, W.Lq, pc.Lp, p.nr_pad, p.w_pad, j, W.red, st));
    GP_CUDA(launch_lz_mnorm_next(S, pc.U, W.R, W.Lq, pc.Lp, p.nr_pad, p.w_pad, j, k, W.red, st));
  }
  GP_CUDA(launch_slq(S, col0, np, k, st));
  return GP_OK;
}

}  // namespace gp

struct HostCg {
  int iters[kMaxW];
  double relres[kMaxW];
};

static gp_status read_cg(const CgState* S, HostCg& h, cudaStream_t st) {
  GP_CUDA(cudaMemcpyAsync(h.iters, S->iters, sizeof(h.iters), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaMemcpyAsync(h.relres, S->relres, sizeof(h.relres), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  return GP_OK;
}

// Common set-up of the solver calls: stage points, build B = [y | Z] (or B = user).
struct SolveSetup {
  SimtPlan pc, pg, pl;
  int slq_prec;
  SolveWs W;
  KernelConsts kc;
  bool precond = false;   // Eq. 1 / Eq. 2 with the Nystrom preconditioner
  Precond pcd;
};

static gp_status setup_solve_plans(const gp_problem* prob, const SolvePlans& P, bool with_grad,
                                   int prec, int lz_k, int slq_prec, void* ws, size_t ws_bytes,
                                   cudaStream_t st, SolveSetup& out) {
  gp_status s;
  const int64_t n = prob->n;
  out.pc = P.pc;
  out.pg = P.pg;
  out.pl = P.pl;
  out.slq_prec = slq_prec;
  SolveWs L = carve_solve(nullptr, P.pc, P.pg, P.pl, with_grad, lz_k, prec, slq_prec);
  if ((s = check_ws(ws, ws_bytes, L.bytes)) != GP_OK) return s;
  out.W = carve_solve(ws, P.pc, P.pg, P.pl, with_grad, lz_k, prec, slq_prec);
  out.kc = kernel_consts(prob);
  GP_CUDA(cudaMemsetAsync(out.W.S, 0, sizeof(CgState), st));
  GP_CUDA(launch_stage_points(prob->X, n, prob->d, prob->d, prob->X, out.kc.csd, out.pc.dp,
                              out.pc.nc_pad, out.W.xs, st));
  GP_CUDA(cudaMemsetAsync(out.W.B, 0, sizeof(float) * out.pc.nr_pad * out.pc.w_pad, st));
  return GP_OK;
}

static gp_status setup_solve(const gp_problem* prob, int w, bool with_grad, int prec, int lz_k,
                             int slq_prec, void* ws, size_t ws_bytes, cudaStream_t st,
                             SolveSetup& out) {
  return setup_solve_plans(prob, solve_plans(prob, w, prec, lz_k, slq_prec), with_grad, prec, lz_k,
                           slq_prec, ws, ws_bytes, st, out);
}

// The arithmetic of the SLQ Lanczos products.
static int slq_prec_of(const gp_solve_opts* o) {
  return o->slq_prec == GP_PREC_SAME ? o->prec : o->slq_prec;
}

static gp_status fill_probes(const gp_problem* prob, const gp_solve_opts* o, float* B, int64_t n_pad,
                             int w_pad, int col_off, cudaStream_t st) {
  if (o->nprobe <= 0) return GP_OK;
  if (o->probes != nullptr) {
    GP_CUDA(launch_pad_block(o->probes, prob->n, o->nprobe, o->nprobe, B, n_pad, w_pad, col_off, st));
  } else {
    GP_CUDA(launch_probes(prob->n, o->nprobe, o->seed, B, w_pad, col_off, n_pad, st));
  }
  return GP_OK;
}

static int effective_maxit(const gp_problem* prob, const gp_solve_opts* o) {
  int64_t m = o->cg_maxit > 0 ? o->cg_maxit : prob->n;
  if (m > 1000000) m = 1000000;
  return static_cast<int>(m);
}

// Bytes of the loss workspace: the solver's, then (precond_rank > 0) the
// preconditioner's planes and factor with its derivative dL/dl.
static size_t loss_bytes(const gp_problem* prob, const gp_solve_opts* o, bool with_grad) {
  const int ww = 1 + o->nprobe;
  const int lz_k = o->nprobe > 0 ? o->nlanczos : 0;
  const int sp = slq_prec_of(o);
  const SolvePlans P = solve_plans(prob, ww, o->prec, lz_k, sp);
  const size_t base = carve_solve(nullptr, P.pc, P.pg, P.pl, with_grad, lz_k, o->prec, sp).bytes;
  if (o->precond_rank <= 0) return base;
  return align256(base) + precond_bytes(P.pc.nr_pad, prob->d, precond_kmax(prob, o->precond_rank),
                                        P.pc.w_pad, lz_k, with_grad);
}

// Forward: CG on [y | Z], SLQ, y^T alpha, loss assembly.  Leaves X = Kh^-1 B.
// With the preconditioner (Eq. 1 / Eq. 2): the factor with dL/dl and the
// closed-form terms first, probes z = L e1 + sqrt(s) e2 ~ N(0, M), PCG, M^-1 of
// the probe block (kept for the gradient pass), SLQ on M^-1/2 Kh M^-1/2 and
// log|M| added to the log-determinant.
static gp_status forward_impl(const gp_problem* prob, const float* y, const gp_solve_opts* o,
                              bool with_grad, void* ws, size_t ws_bytes, cudaStream_t st,
                              SolveSetup& ss, gp_status& cg_status) {
  gp_status s;
  const int p = o->nprobe;
  const int w = 1 + p;
  const int lz_k = p > 0 ? o->nlanczos : 0;
  const bool precond = o->precond_rank > 0;
  if (precond && (s = check_ws(ws, ws_bytes, loss_bytes(prob, o, with_grad))) != GP_OK) return s;
  if ((s = setup_solve(prob, w, with_grad, o->prec, lz_k, slq_prec_of(o), ws, ws_bytes, st, ss)) !=
      GP_OK)
    return s;
  SolveWs& W = ss.W;
  const int64_t n = prob->n;
  ss.precond = precond;
  if (precond) {
    const int kmax = precond_kmax(prob, o->precond_rank);
    ss.pcd = carve_precond(static_cast<char*>(ws) + align256(W.bytes), ss.pc.nr_pad, prob->d, kmax,
                           ss.pc.w_pad, lz_k, with_grad);
    set_live_width(ss.pcd, w);
    if ((s = build_precond(prob, kmax, o->precond_tol, ss.pcd, st)) != GP_OK) return s;
    GP_CUDA(nys_closed_terms(ss.pcd.ws, ss.pcd.rank, n, prob->theta.s, prob->theta.f,
                             &W.S->logdet_m, W.S->trm, st));
  }
  GP_CUDA(launch_pad_block(y, n, 1, 1, W.B, ss.pc.nr_pad, ss.pc.w_pad, 0, st));
  if (precond) {
    if (p > 0)
      GP_CUDA(nys_probes(ss.pcd.ws, ss.pcd.rank, n, prob->theta.s, o->probes, o->seed, p, W.B, 1, st));
  } else if ((s = fill_probes(prob, o, W.B, ss.pc.nr_pad, ss.pc.w_pad, 1, st)) != GP_OK) {
    return s;
  }
  s = run_cg(prob, ss.pc, o->prec, W, w, effective_maxit(prob, o), o->cg_rtol, st,
             precond ? &ss.pcd : nullptr);
  if (s != GP_OK) return s;
  if (p > 0) {
    if (precond) {
      GP_CUDA(nys_apply(ss.pcd.ws, ss.pcd.rank, n, ss.pcd.s, W.B, ss.pcd.Z, nullptr, st));
      if ((s = run_lanczos_m(prob, ss.pl, ss.slq_prec, W, ss.pcd, 1, p, o->nlanczos, st)) != GP_OK)
        return s;
    } else if ((s = run_lanczos(prob, ss.pl, ss.slq_prec, W, 1, p, o->nlanczos, st)) != GP_OK) {
      return s;
    }
    GP_CUDA(cudaMemcpyAsync(W.S->out, W.S2->out, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  if (precond) GP_CUDA(launch_add_logdet_m(W.S, st));
  GP_CUDA(launch_yalpha(W.S, W.B, W.X, ss.pc.nr_pad, ss.pc.w_pad, W.red, st));
  GP_CUDA(launch_assemble(W.S, prob->n, p, st));
  cg_status = GP_OK;
  return GP_OK;
}

// Backward: fused product with V = [alpha | Z] against W = X; gradient assembly.
static gp_status backward_impl(const gp_problem* prob, const gp_solve_opts* o, SolveSetup& ss,
                               cudaStream_t st) {
  gp_status s;
  SolveWs& W = ss.W;
  const int p = o->nprobe;
  const int w = 1 + p;
  const SimtPlan& pg = ss.pg;
  // V = B with column 0 replaced by alpha (reuse Q as V); with the
  // preconditioner, V = [alpha | M^-1 Z] (Eq. 2's Hutchinson terms with z ~ N(0, M)).
  GP_CUDA(cudaMemcpyAsync(W.Q, ss.precond ? ss.pcd.Z : W.B, sizeof(float) * pg.nr_pad * pg.w_pad,
                          cudaMemcpyDeviceToDevice, st));
  GP_CUDA(launch_copy_col0(W.X, W.Q, pg.nr_pad, pg.w_pad, st));
  if (ss.kc.ard) {
    // Per-dimension length-scales: the s terms from column dot products, the f
    // and l_t terms from one fused contraction of the entries with Gq and Gt.
    GP_CUDA(launch_coldots(W.S, W.X, W.Q, pg.nr_pad, pg.w_pad, w, W.red, st));
    const GradArdPlan g = plan_grad_ard(pg.nr_pad, prob->d);
    ArdScales c{};
    for (int t = 0; t < prob->d; ++t) c.v[t] = ss.kc.ct[t];
    const cudaError_t e = launch_grad_ard(g, prob->kernel, w, p, prob->d, pg.dp, W.xs, W.Q, W.X,
                                          pg.nr_pad, pg.w_pad, reinterpret_cast<double*>(W.part),
                                          W.S, prob->theta.f, c, st);
    if (e == cudaErrorNotSupported)
      return fail(GP_ERR_UNIMPLEMENTED, "per-dimension length-scales need 1 + nprobe <= 48");
    if (e != cudaSuccess) return cuda_fail(e, "launch_grad_ard");
    return GP_OK;
  }
  float* part_k = W.part;
  float* part_d = W.part + static_cast<size_t>(pg.split) * pg.nr_pad * pg.w_pad;
  if ((s = run_product(pg, prob->kernel, true, GP_PREC_FP32, W.xs, W.xs, W.Q, nullptr, part_k, part_d,
                       nullptr, &W.S->err, st)) != GP_OK)
    return s;
  const double f = prob->theta.f;
  GP_CUDA(launch_grad_dots(W.S, part_k, part_d, pg.split, W.Q, W.X, pg.nr_pad, pg.w_pad, w, 2.0 * f,
                           f * f * ss.kc.cD, W.red, st));
  if (ss.precond && p > 0) {
    // Subtract v^T (dM/dtheta) v, v = M^-1 z: v^T v, (2/f) |L^T v|^2, 2 (L^T v).(dL^T v).
    GP_CUDA(launch_plane_dots(W.S, W.Q, W.Q, pg.nr_pad, pg.w_pad, W.S->vv, W.red, st));
    GP_CUDA(nys_lt_times(ss.pcd.ws, ss.pcd.rank, false, W.Q, ss.pcd.ws.U, st));
    GP_CUDA(nys_lt_times(ss.pcd.ws, ss.pcd.rank, true, W.Q, ss.pcd.ws.U2, st));
    GP_CUDA(launch_precond_corr(W.S, ss.pcd.ws.U, ss.pcd.ws.U2, ss.pcd.rank, pg.w_pad, p, f, st));
  }
  GP_CUDA(launch_assemble(W.S, prob->n, p, st));
  return GP_OK;
}

static gp_status read_outputs(const CgState* S, const CgState* S2, int w, double out[16],
                              gp_loss_info* info, cudaStream_t st) {
  HostCg h;
  gp_status s;
  if ((s = read_cg(S, h, st)) != GP_OK) return s;
  GP_CUDA(cudaMemcpyAsync(out, S->out, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  double mterms[4];
  GP_CUDA(cudaMemcpyAsync(mterms, &S->logdet_m, sizeof(mterms), cudaMemcpyDeviceToHost, st));
  int err = 0, err2 = 0;
  GP_CUDA(cudaMemcpyAsync(&err, &S->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (S2 != nullptr)
    GP_CUDA(cudaMemcpyAsync(&err2, &S2->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  if (err == 0) err = err2;
  if (info != nullptr) {
    info->yalpha = out[15];
    info->logdet = out[0];
    info->logdet_stderr = out[1];
    for (int t = 0; t < 3; ++t) {
      info->quad[t] = out[6 + t];
      info->trace[t] = out[9 + t];
      info->trace_stderr[t] = out[12 + t];
    }
    int mx = 0;
    double rmax = 0.0;
    for (int c = 0; c < w; ++c) {
      mx = std::max(mx, h.iters[c]);
      rmax = std::max(rmax, h.relres[c]);
    }
    info->cg_iters = mx;
    info->refine_steps = 0;
    info->relres_y = h.relres[0];
    info->relres_max = rmax;
    info->logdet_m = mterms[0];
    for (int t = 0; t < 3; ++t) info->trace_m[t] = mterms[1 + t];
  }
  if (err == kDevTimeout) return fail(GP_ERR_TIMEOUT, "a bounded device wait gave up");
  if (err == kDevBreakdown) return fail(GP_ERR_BREAKDOWN, "CG breakdown");
  if (err == kDevNumeric) return fail(GP_ERR_NUMERIC, "non-positive Lanczos eigenvalue");
  return GP_OK;
}

static gp_status check_conv(const CgState* S, int w, int maxit, double rtol, cudaStream_t st) {
  HostCg h;
  gp_status s;
  if ((s = read_cg(S, h, st)) != GP_OK) return s;
  for (int c = 0; c < w; ++c)
    if (h.relres[c] > rtol && h.iters[c] >= maxit)
      return fail(GP_ERR_NOT_CONVERGED, "CG reached cg_maxit before cg_rtol (column " +
                                            std::to_string(c) + ", relres " +
                                            std::to_string(h.relres[c]) + ")");
  return GP_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision iterative refinement.  Outer loop: r = B - Kh x with x in
// FP64 and the O(n^2 w) sums in FP32-pair arithmetic (or FP64, on request);
// stop when ||r_c|| / ||B_c|| <= refine_rtol for every column.  Inner loop:
// block CG on the product of arithmetic opts->prec for Kh d = r to
// opts->cg_rtol; x += d.
// Workspace: the solver workspace of the inner CG, then x (FP64), r (FP64),
// the padded right-hand side (FP32), the residual's split partial sums (FP64)
// and its error word.
// ---------------------------------------------------------------------------
static size_t refine_extra_offset(const SimtPlan& pc, int prec) {
  return (carve_solve(nullptr, pc, pc, pc, false, 0, prec, prec).bytes + 255) &
         ~static_cast<size_t>(255);
}

static size_t refine_bytes(const SimtPlan& pc, int prec, int64_t n, int w) {
  const size_t plane = static_cast<size_t>(pc.nr_pad) * pc.w_pad;
  size_t off = refine_extra_offset(pc, prec) + 2 * plane * sizeof(double) + plane * sizeof(float);
  off = (off + 255) & ~static_cast<size_t>(255);
  return off + residual_part_bytes_bound(n, w) + 1024;
}

// Workspace of the residual calls: x (FP64), r (FP64), padded B, padded X and
// the FP32 residual (all [n_pad][w_pad]), reduction scratch, one CgState, the
// split partial sums of the residual kernel and an error word.
struct ResidualWs {
  double* x64;
  double* r64;
  float* Bp;
  float* Xp;
  float* rf;
  double* red;
  CgState* S;
  double* part;
  int* err;
  size_t bytes;
};

static ResidualWs carve_residual(void* ws, int64_t n, int w) {
  const int64_t n_pad = round_up(n, kPad);
  const int w_pad = static_cast<int>(round_up(w, 4));
  Carve c(ws);
  ResidualWs r;
  const size_t plane = static_cast<size_t>(n_pad) * w_pad;
  r.x64 = c.take<double>(plane);
  r.r64 = c.take<double>(plane);
  r.Bp = c.take<float>(plane);
  r.Xp = c.take<float>(plane);
  r.rf = c.take<float>(plane);
  r.red = c.take<double>(red_doubles(n_pad, w_pad));
  r.S = c.take<CgState>(1);
  r.part = c.take<double>(residual_part_bytes_bound(n, w) / sizeof(double));
  r.err = c.take<int>(64);
  r.bytes = c.off + 256;
  return r;
}

static int residual_arith(int abi) { return abi == GP_RESIDUAL_FP64 ? kResF64 : kResPair; }

// R = B - Kh x64 over rows (NULL: 0..m-1) into the padded plane R [m_pad][ldr];
// Bg (may be NULL) receives the B rows in the same layout.
static gp_status residual_into(const gp_problem* prob, const float* B, int64_t ldb, const double* x64,
                               int64_t ldx, int w, const int64_t* rows, int64_t m, int arith,
                               double* part, int* err, double* R, int ldr, float* Bg,
                               cudaStream_t st) {
  const ResPlan p = plan_residual(m, prob->n, w);
  ResArgs a{};
  a.X = prob->X;
  a.n = prob->n;
  a.d = prob->d;
  a.kernel = prob->kernel;
  a.rows = rows;
  a.m = m;
  a.x64 = x64;
  a.ldx = ldx;
  a.w = w;
  a.part = part;
  const double l = prob->theta.l;
  a.kc64 = prob->kernel == GP_KERNEL_GAUSSIAN ? 1.0 / (2.0 * l * l) : sqrt(3.0) / l;
  a.kc = pa::kernel_pair_const(prob->kernel, l);
  a.err = err;
  ResidualCall c{arith, B, ldb, prob->theta.f * prob->theta.f, prob->theta.s, R, ldr, Bg};
  GP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  GP_CUDA(launch_residual(p, a, c, st));
  return GP_OK;
}

gp_status refine_solve(const gp_problem* prob, const float* B, int32_t w, float* Xsol, double* X64,
                       const gp_solve_opts* opts, int32_t* iters, double* relres, void* ws,
                       size_t ws_bytes, cudaStream_t st) {
  gp_status s;
  const int64_t n = prob->n;
  const int prec = opts->prec;
  SimtPlan pc = plan_for(n, n, prob->d, w, false, prob->kernel, prec);
  SimtPlan pg = plan_for(n, n, prob->d, w, true, prob->kernel, GP_PREC_FP32);
  unify_width(pc, pg);   // the widths setup_solve uses
  const size_t base = refine_bytes(pc, prec, n, w);
  const int kmax = precond_kmax(prob, opts->precond_rank);
  const size_t need = kmax > 0 ? align256(base) + precond_bytes(pc.nr_pad, prob->d, kmax, pc.w_pad) : base;
  if ((s = check_ws(ws, ws_bytes, need)) != GP_OK) return s;
  SolveSetup ss;
  if ((s = setup_solve(prob, w, false, prec, 0, prec, ws, ws_bytes, st, ss)) != GP_OK) return s;
  Precond pcond;
  if (kmax > 0) {
    pcond = carve_precond(static_cast<char*>(ws) + align256(base), ss.pc.nr_pad, prob->d, kmax,
                          ss.pc.w_pad);
    set_live_width(pcond, w);
    if ((s = build_precond(prob, kmax, opts->precond_tol, pcond, st)) != GP_OK) return s;
  }
  const size_t plane = static_cast<size_t>(ss.pc.nr_pad) * ss.pc.w_pad;
  char* extra = static_cast<char*>(ws) + refine_extra_offset(ss.pc, prec);
  double* x64 = reinterpret_cast<double*>(extra);
  double* r64 = x64 + plane;
  float* Bp = reinterpret_cast<float*>(r64 + plane);
  const size_t part_off =
      ((refine_extra_offset(ss.pc, prec) + 2 * plane * sizeof(double) + plane * sizeof(float)) + 255) &
      ~static_cast<size_t>(255);
  double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + part_off);
  int* rerr = reinterpret_cast<int*>(reinterpret_cast<char*>(part) + residual_part_bytes_bound(n, w));
  const int arith = residual_arith(opts->refine_residual);
  GP_CUDA(cudaMemsetAsync(x64, 0, 2 * plane * sizeof(double), st));
  GP_CUDA(cudaMemsetAsync(Bp, 0, plane * sizeof(float), st));
  GP_CUDA(cudaMemsetAsync(ss.W.S2, 0, sizeof(CgState), st));
  GP_CUDA(launch_pad_block(B, n, w, w, Bp, ss.pc.nr_pad, ss.pc.w_pad, 0, st));
  const int max_outer = opts->refine_maxit > 0 ? opts->refine_maxit : 10;
  const int inner_maxit = effective_maxit(prob, opts);
  std::vector<int> total_iters(w, 0);
  HostCg hr;
  for (int outer = 0;; ++outer) {
    if (outer == 0) {
      // x = 0: the residual is B itself (no O(n^2) pass).
      GP_CUDA(launch_widen(Bp, r64, static_cast<int64_t>(plane), st));
    } else if ((s = residual_into(prob, Bp, ss.pc.w_pad, x64, ss.pc.w_pad, w, nullptr, n, arith, part,
                                  rerr, r64, ss.pc.w_pad, nullptr, st)) != GP_OK) {
      return s;
    }
    GP_CUDA(launch_refine_norms(ss.W.S2, r64, Bp, ss.W.B, ss.pc.nr_pad, ss.pc.w_pad, w, ss.W.red, st));
    if ((s = read_cg(ss.W.S2, hr, st)) != GP_OK) return s;
    bool done = true;
    for (int c = 0; c < w; ++c) done = done && !(hr.relres[c] > opts->refine_rtol);
    if (done || outer >= max_outer) break;
    if ((s = run_cg(prob, ss.pc, prec, ss.W, w, inner_maxit, opts->cg_rtol, st,
                    kmax > 0 ? &pcond : nullptr)) != GP_OK)
      return s;
    HostCg hi;
    if ((s = read_cg(ss.W.S, hi, st)) != GP_OK) return s;
    for (int c = 0; c < w; ++c) total_iters[c] += hi.iters[c];
    GP_CUDA(launch_refine_update(x64, ss.W.X, ss.pc.nr_pad, ss.pc.w_pad, w, st));
  }
  if (Xsol != nullptr) GP_CUDA(launch_refine_out(x64, Xsol, n, ss.pc.w_pad, w, st));
  if (X64 != nullptr)
    GP_CUDA(cudaMemcpy2DAsync(X64, sizeof(double) * w, x64, sizeof(double) * ss.pc.w_pad,
                              sizeof(double) * w, n, cudaMemcpyDeviceToDevice, st));
  GP_CUDA(cudaStreamSynchronize(st));
  bool conv = true;
  for (int c = 0; c < w; ++c) {
    if (iters) iters[c] = total_iters[c];
    if (relres) relres[c] = hr.relres[c];
    conv = conv && !(hr.relres[c] > opts->refine_rtol);
  }
  if (!conv) return fail(GP_ERR_NOT_CONVERGED, "refinement reached refine_maxit before refine_rtol");
  return GP_OK;
}

// ---------------------------------------------------------------------------
// Batched loss and gradient: several problems advanced together, with one
// grouped product launch (kmv_simt_group_kernel) per CG iteration, per
// Lanczos step and for the gradient pass, covering every member; the O(n w)
// steps stay per member.  FP32 products; the widths are padded up to a
// grouped TW (batch_plans), so every member shares one instantiation.
// ---------------------------------------------------------------------------
namespace {

int group_tw(int tw) {
  for (int t : kGroupTW)
    if (t >= tw) return t;
  return 0;
}

SolvePlans batch_plans(const gp_problem* prob, int w, int lz_k) {
  SolvePlans P = solve_plans(prob, w, GP_PREC_FP32, lz_k, GP_PREC_FP32);
  const int tw = group_tw(P.pc.tw);
  for (SimtPlan* q : {&P.pc, &P.pg, &P.pl}) {
    q->tw = tw;
    q->w_pad = q->ng * tw;
  }
  return P;
}

struct BatchMember {
  const gp_problem* prob;
  const float* y;
  const gp_solve_opts* o;
  void* ws;
  size_t ws_bytes;
  SolveSetup ss;
  gp_status status = GP_OK;
};

enum class GroupPhase { kCg, kLanczos, kGrad };

// One grouped product over the members (in the given order); members whose
// active flag is 0 are skipped on the device.
gp_status group_product(std::vector<BatchMember*>& M, GroupPhase ph, int j, cudaStream_t st) {
  SimtGroup g{};
  g.count = static_cast<int>(M.size());
  g.counter = &M[0]->ss.W.S->group_counter;
  int items = 0;
  for (int k = 0; k < g.count; ++k) {
    SolveSetup& ss = M[k]->ss;
    SolveWs& W = ss.W;
    const SimtPlan& p = ph == GroupPhase::kGrad ? ss.pg : (ph == GroupPhase::kLanczos ? ss.pl : ss.pc);
    const size_t plane = static_cast<size_t>(p.nr_pad) * p.w_pad;
    SimtArgs a{W.xs, W.xs, W.P, W.part, nullptr, &W.S->n_active, &W.S->err};
    if (ph == GroupPhase::kLanczos) {
      a.v = W.Lq + static_cast<size_t>(j) * plane;
      a.active = &W.S2->n_active;
      a.err = &W.S2->err;
    } else if (ph == GroupPhase::kGrad) {
      a.v = W.Q;
      a.part_d = W.part + static_cast<size_t>(p.split) * plane;
      a.active = nullptr;
    }
    g.e[k] = SimtGroupEntry{a, p.nr_pad, p.row_tiles, p.split, p.jtiles, p.jt_per_split, items};
    items += p.row_tiles * p.split;
  }
  g.total_items = items;
  const SimtPlan& p0 = ph == GroupPhase::kGrad ? M[0]->ss.pg : M[0]->ss.pc;
  GP_CUDA(cudaMemsetAsync(g.counter, 0, sizeof(int), st));
  profile_product_begin(st);
  const cudaError_t e =
      launch_simt_group(p0, M[0]->prob->kernel, ph == GroupPhase::kGrad, g, st);
  profile_product_end(st);
  if (e != cudaSuccess) return cuda_fail(e, "launch_simt_group");
  return GP_OK;
}

// One CG iteration of every member: the grouped product, then each member's
// O(n w) step (fused cooperative launch where it fits).
gp_status batch_cg_iteration(std::vector<BatchMember*>& M, cudaStream_t st) {
  gp_status s;
  if ((s = group_product(M, GroupPhase::kCg, 0, st)) != GP_OK) return s;
  for (BatchMember* m : M) {
    const gp_problem* prob = m->prob;
    const SimtPlan& p = m->ss.pc;
    SolveWs& W = m->ss.W;
    const double f2 = prob->theta.f * prob->theta.f;
    if (thread_cooperative() && cg_fused_wanted() && cg_step_fits(p.nr_pad)) {
      GP_CUDA(launch_cg_step(W.S, W.part, p.split, W.X, W.R, W.P, W.Q, p.nr_pad, prob->n, p.w_pad,
                             f2, prob->theta.s, W.red, st));
    } else {
      GP_CUDA(launch_cg_epi_alpha(W.S, W.part, p.split, W.P, W.Q, p.nr_pad, prob->n, p.w_pad, f2,
                                  prob->theta.s, W.red, st));
      GP_CUDA(launch_cg_update(W.S, W.X, W.R, W.P, W.Q, p.nr_pad, p.w_pad, W.red, st));
      GP_CUDA(launch_cg_pupdate(W.S, W.R, W.P, p.nr_pad, p.w_pad, st));
    }
  }
  return GP_OK;
}

gp_status batch_run_cg(std::vector<BatchMember*>& M, int maxit, cudaStream_t st) {
  for (BatchMember* m : M) {
    const SimtPlan& p = m->ss.pc;
    SolveWs& W = m->ss.W;
    GP_CUDA(launch_cg_init(W.S, W.B, W.X, W.R, W.P, p.nr_pad, p.w_pad, 1 + m->o->nprobe,
                           effective_maxit(m->prob, m->o), m->o->cg_rtol, W.red, st));
  }
  std::vector<int> h(2 * M.size());
  IterationGraph graph;
  bool tried = false, use_graph = false;
  int chunk = 4, issued = 0;
  while (issued < maxit) {
    const int todo = std::min(chunk, maxit - issued);
    for (int k = 0; k < todo; ++k) {
      if (issued + k > 0 && !tried) {
        tried = true;
        use_graph = graph.capture([&](cudaStream_t cs) { return batch_cg_iteration(M, cs); });
      }
      if (use_graph) {
        GP_CUDA(graph.launch(st));
      } else {
        gp_status s = batch_cg_iteration(M, st);
        if (s != GP_OK) return s;
      }
    }
    issued += todo;
    for (size_t k = 0; k < M.size(); ++k)
      GP_CUDA(cudaMemcpyAsync(&h[2 * k], M[k]->ss.W.S, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GP_CUDA(cudaStreamSynchronize(st));
    bool any = false;
    for (size_t k = 0; k < M.size(); ++k) {
      if (h[2 * k + 1] == kDevTimeout) return fail(GP_ERR_TIMEOUT, "a bounded device wait gave up");
      any = any || (h[2 * k] != 0 && h[2 * k + 1] == 0);
    }
    if (!any) break;
    if (chunk < 32) chunk *= 2;
  }
  return GP_OK;
}

gp_status batch_run_lanczos(std::vector<BatchMember*>& M, int np, int k, cudaStream_t st) {
  gp_status s;
  for (BatchMember* m : M) {
    const SimtPlan& p = m->ss.pl;
    SolveWs& W = m->ss.W;
    GP_CUDA(cudaMemsetAsync(W.S2, 0, sizeof(CgState), st));
    GP_CUDA(launch_lz_init(W.S2, W.B, W.Lq, p.nr_pad, p.w_pad, 1, np, W.red, st));
  }
  for (int j = 0; j < k; ++j) {
    if ((s = group_product(M, GroupPhase::kLanczos, j, st)) != GP_OK) return s;
    for (BatchMember* m : M) {
      const gp_problem* prob = m->prob;
      const SimtPlan& p = m->ss.pl;
      SolveWs& W = m->ss.W;
      CgState* S = W.S2;
      const float* Qj = W.Lq + static_cast<size_t>(j) * p.nr_pad * p.w_pad;
      GP_CUDA(launch_lz_epi_alpha(S, W.part, p.split, Qj, W.R, p.nr_pad, prob->n, p.w_pad,
                                  prob->theta.f * prob->theta.f, prob->theta.s, j, W.red, st));
      GP_CUDA(launch_lz_three_term(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, st));
      GP_CUDA(launch_lz_reorth(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, W.red, st));
      GP_CUDA(launch_lz_reorth(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, W.red, st));
      GP_CUDA(launch_lz_norm_next(S, W.R, W.Lq, p.nr_pad, p.w_pad, j, k, W.red, st));
    }
  }
  for (BatchMember* m : M) {
    SolveWs& W = m->ss.W;
    GP_CUDA(launch_slq(W.S2, 1, np, k, st));
    GP_CUDA(cudaMemcpyAsync(W.S->out, W.S2->out, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return GP_OK;
}

gp_status check_batch(int32_t count, const gp_problem* probs, const float* const* ys,
                      const gp_solve_opts* opts) {
  gp_status s;
  if (count < 1 || count > kMaxGroup) return fail(GP_ERR_ARG, "count must be in [1, 64]");
  if (probs == nullptr || ys == nullptr || opts == nullptr)
    return fail(GP_ERR_ARG, "probs, y and opts must be non-NULL");
  for (int k = 0; k < count; ++k) {
    if ((s = check_problem(&probs[k])) != GP_OK) return s;
    if ((s = check_opts(&opts[k], false)) != GP_OK) return s;
    if (ys[k] == nullptr) return fail(GP_ERR_ARG, "y[k] is NULL");
    if (probs[k].ls != nullptr)
      return fail(GP_ERR_UNIMPLEMENTED, "batched solves take isotropic length-scales");
    if (opts[k].prec != GP_PREC_FP32 || slq_prec_of(&opts[k]) != GP_PREC_FP32)
      return fail(GP_ERR_UNIMPLEMENTED, "batched solves use FP32 products");
    if (1 + opts[k].nprobe > 64) return fail(GP_ERR_UNIMPLEMENTED, "batched solves need 1 + nprobe <= 64");
    if (probs[k].kernel != probs[0].kernel || dim_template(probs[k].d) != dim_template(probs[0].d))
      return fail(GP_ERR_ARG, "batch members must share the kernel and the dimension template");
    if (opts[k].nprobe != opts[0].nprobe || opts[k].nlanczos != opts[0].nlanczos)
      return fail(GP_ERR_ARG, "batch members must share nprobe and nlanczos");
  }
  return GP_OK;
}

}  // namespace

static gp_status loss_and_grad_batch(int32_t count, const gp_problem* probs, const float* const* ys,
                                     const gp_solve_opts* opts, double* loss, double* grad,
                                     gp_loss_info* info, int32_t* status, void* const* ws,
                                     const size_t* ws_bytes, cudaStream_t st) {
  gp_status s;
  if ((s = check_batch(count, probs, ys, opts)) != GP_OK) return s;
  if (ws == nullptr || ws_bytes == nullptr) return fail(GP_ERR_ARG, "ws and ws_bytes must be non-NULL");
  std::vector<BatchMember> mem(count);
  const int p = opts[0].nprobe;
  const int w = 1 + p;
  const int lz_k = p > 0 ? opts[0].nlanczos : 0;
  int maxit = 0;
  for (int k = 0; k < count; ++k) {
    BatchMember& m = mem[k];
    m.prob = &probs[k];
    m.y = ys[k];
    m.o = &opts[k];
    const SolvePlans P = batch_plans(m.prob, w, lz_k);
    if ((s = setup_solve_plans(m.prob, P, true, GP_PREC_FP32, lz_k, GP_PREC_FP32, ws[k],
                               ws_bytes[k], st, m.ss)) != GP_OK)
      return s;
    SolveWs& W = m.ss.W;
    GP_CUDA(launch_pad_block(m.y, m.prob->n, 1, 1, W.B, m.ss.pc.nr_pad, m.ss.pc.w_pad, 0, st));
    if ((s = fill_probes(m.prob, m.o, W.B, m.ss.pc.nr_pad, m.ss.pc.w_pad, 1, st)) != GP_OK) return s;
    maxit = std::max(maxit, effective_maxit(m.prob, m.o));
  }
  // Largest problems first, so that the persistent CTAs start on the longest items.
  std::vector<BatchMember*> M;
  for (BatchMember& m : mem) M.push_back(&m);
  std::stable_sort(M.begin(), M.end(),
                   [](const BatchMember* a, const BatchMember* b) { return a->prob->n > b->prob->n; });
  // The loop runs to the largest cg_maxit; each member's state carries its own
  // cap, after which its columns are inactive and its tiles are skipped.
  if ((s = batch_run_cg(M, maxit, st)) != GP_OK) return s;
  if (p > 0 && (s = batch_run_lanczos(M, p, opts[0].nlanczos, st)) != GP_OK) return s;
  for (BatchMember* m : M) {
    SolveWs& W = m->ss.W;
    const SimtPlan& pc = m->ss.pc;
    GP_CUDA(launch_yalpha(W.S, W.B, W.X, pc.nr_pad, pc.w_pad, W.red, st));
    GP_CUDA(launch_assemble(W.S, m->prob->n, p, st));
    // Gradient pass operands: V = B with column 0 replaced by alpha.
    const SimtPlan& pg = m->ss.pg;
    GP_CUDA(cudaMemcpyAsync(W.Q, W.B, sizeof(float) * pg.nr_pad * pg.w_pad, cudaMemcpyDeviceToDevice,
                            st));
    GP_CUDA(launch_copy_col0(W.X, W.Q, pg.nr_pad, pg.w_pad, st));
  }
  if ((s = group_product(M, GroupPhase::kGrad, 0, st)) != GP_OK) return s;
  for (BatchMember* m : M) {
    SolveWs& W = m->ss.W;
    const SimtPlan& pg = m->ss.pg;
    const double f = m->prob->theta.f;
    float* part_k = W.part;
    float* part_d = W.part + static_cast<size_t>(pg.split) * pg.nr_pad * pg.w_pad;
    GP_CUDA(launch_grad_dots(W.S, part_k, part_d, pg.split, W.Q, W.X, pg.nr_pad, pg.w_pad, w,
                             2.0 * f, f * f * m->ss.kc.cD, W.red, st));
    GP_CUDA(launch_assemble(W.S, m->prob->n, p, st));
  }
  gp_status worst = GP_OK;
  for (int k = 0; k < count; ++k) {
    BatchMember& m = mem[k];
    double out[16];
    gp_status sk = read_outputs(m.ss.W.S, p > 0 ? m.ss.W.S2 : nullptr, w, out,
                                info ? &info[k] : nullptr, st);
    if (sk == GP_OK) {
      if (loss) loss[k] = out[2];
      if (grad)
        for (int t = 0; t < 3; ++t) grad[3 * k + t] = out[3 + t];
      sk = check_conv(m.ss.W.S, w, effective_maxit(m.prob, m.o), m.o->cg_rtol, st);
    }
    if (status) status[k] = sk;
    if (sk != GP_OK && (worst == GP_OK || worst == GP_ERR_NOT_CONVERGED)) worst = sk;
  }
  if (worst == GP_ERR_NOT_CONVERGED)
    return fail(GP_ERR_NOT_CONVERGED, "a batch member reached cg_maxit before cg_rtol");
  return worst;
}

// ---------------------------------------------------------------------------
// Exported entry points.
// ---------------------------------------------------------------------------
extern "C" {

const char* gp_version(void) { return "libgp 0.1 (sm_103a)"; }

const char* gp_last_error(void) { return last_error_cstr(); }

const char* gp_status_string(gp_status st) {
  switch (st) {
    case GP_OK: return "GP_OK";
    case GP_ERR_ARG: return "GP_ERR_ARG";
    case GP_ERR_CUDA: return "GP_ERR_CUDA";
    case GP_ERR_OOM: return "GP_ERR_OOM";
    case GP_ERR_NOT_CONVERGED: return "GP_ERR_NOT_CONVERGED";
    case GP_ERR_BREAKDOWN: return "GP_ERR_BREAKDOWN";
    case GP_ERR_TIMEOUT: return "GP_ERR_TIMEOUT";
    case GP_ERR_UNIMPLEMENTED: return "GP_ERR_UNIMPLEMENTED";
    case GP_ERR_NUMERIC: return "GP_ERR_NUMERIC";
  }
  return "GP_ERR_UNKNOWN";
}

size_t gp_workspace_bytes(gp_op op, const gp_problem* prob, int32_t w, const gp_solve_opts* opts) {
  if (check_problem(prob) != GP_OK) return 0;
  const int64_t n = prob->n;
  const int prec = opts != nullptr ? opts->prec : GP_PREC_FP32;
  switch (op) {
    case GP_OP_MATMUL:
    case GP_OP_GRAD_MATMUL: {
      if (check_width(w) != GP_OK) return 0;
      const bool grad = op == GP_OP_GRAD_MATMUL;
      return carve_product(nullptr, plan_for(n, n, prob->d, w, grad, prob->kernel, prec), grad, false, prec)
          .bytes;
    }
    case GP_OP_PREDICT: {
      if (w < 1) {
        set_error("predict: m must be >= 1");
        return 0;
      }
      return carve_product(nullptr, plan_for(w, n, prob->d, 1, false, prob->kernel, GP_PREC_FP32),
                           false, true, GP_PREC_FP32)
          .bytes;
    }
    case GP_OP_RESIDUAL: {
      if (check_width(w) != GP_OK) return 0;
      return carve_residual(nullptr, n, w).bytes;
    }
    case GP_OP_LOSS_GRAD_BATCH: {
      if (check_opts(opts, false) != GP_OK) return 0;
      if (1 + opts->nprobe > 64) {
        set_error("batched solves need 1 + nprobe <= 64");
        return 0;
      }
      const int lz_k = opts->nprobe > 0 ? opts->nlanczos : 0;
      const SolvePlans P = batch_plans(prob, 1 + opts->nprobe, lz_k);
      return carve_solve(nullptr, P.pc, P.pg, P.pl, true, lz_k, GP_PREC_FP32, GP_PREC_FP32).bytes;
    }
    case GP_OP_PREDICT_VAR: {
      if (w < 1) {
        set_error("predict_var: m must be >= 1");
        return 0;
      }
      const int wb = static_cast<int>(std::min<int64_t>(w, GP_MAX_COLS));
      const SolvePlans P = solve_plans(prob, wb, prec, 0, prec);
      return carve_solve(nullptr, P.pc, P.pg, P.pl, false, 0, prec, prec).bytes;
    }
    case GP_OP_PCG: {
      if (check_width(w) != GP_OK) return 0;
      SimtPlan pc = plan_for(n, n, prob->d, w, false, prob->kernel, prec);
      SimtPlan pg = plan_for(n, n, prob->d, w, true, prob->kernel, GP_PREC_FP32);
      unify_width(pc, pg);
      const size_t base = opts != nullptr && opts->refine_rtol > 0
                              ? refine_bytes(pc, prec, n, w)
                              : carve_solve(nullptr, pc, pc, pc, false, 0, prec, prec).bytes;
      if (opts == nullptr || opts->precond_rank == 0) return base;
      if (check_opts(opts, false, true) != GP_OK) return 0;
      return align256(base) +
             precond_bytes(pc.nr_pad, prob->d, precond_kmax(prob, opts->precond_rank), pc.w_pad);
    }
    case GP_OP_NYSTROM: {
      if (check_width(w) != GP_OK) return 0;
      if (opts == nullptr || opts->precond_rank < 1 || opts->precond_rank > GP_MAX_PRECOND_RANK) {
        set_error("GP_OP_NYSTROM needs opts->precond_rank in [1, 4096]");
        return 0;
      }
      return nystrom_entry_bytes(prob, w, precond_kmax(prob, opts->precond_rank));
    }
    case GP_OP_SLQ:
    case GP_OP_LOSS_GRAD: {
      if (check_opts(opts, op == GP_OP_SLQ, op == GP_OP_LOSS_GRAD) != GP_OK) return 0;
      if (op == GP_OP_LOSS_GRAD) return loss_bytes(prob, opts, true);
      const int ww = op == GP_OP_SLQ ? opts->nprobe : 1 + opts->nprobe;
      const int lz_k = opts->nprobe > 0 ? opts->nlanczos : 0;
      const int sp = slq_prec_of(opts);
      const SolvePlans P = solve_plans(prob, ww, prec, lz_k, sp);
      return carve_solve(nullptr, P.pc, P.pg, P.pl, op == GP_OP_LOSS_GRAD, lz_k, prec, sp).bytes;
    }
  }
  set_error("unknown op");
  return 0;
}

gp_status gp_kernel_matmul(const gp_problem* prob, const float* V, int32_t w, float* Y, int32_t prec,
                           void* ws, size_t ws_bytes, void* stream) {
  return product_call(prob, V, w, Y, nullptr, nullptr, false, prec, ws, ws_bytes, stream);
}

gp_status gp_kernel_grad_matmul(const gp_problem* prob, const float* V, int32_t w, float* Y,
                                float* dY_f, float* dY_l, int32_t prec, void* ws, size_t ws_bytes,
                                void* stream) {
  return product_call(prob, V, w, Y, dY_f, dY_l, true, prec, ws, ws_bytes, stream);
}

gp_status gp_pcg_solve(const gp_problem* prob, const float* B, int32_t w, float* Xsol,
                       const gp_solve_opts* opts, int32_t* iters, double* relres, void* ws,
                       size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_width(w)) != GP_OK) return s;
  if ((s = check_opts(opts, false, true)) != GP_OK) return s;
  if (B == nullptr || Xsol == nullptr) return fail(GP_ERR_ARG, "B and Xsol must be non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (opts->prec != GP_PREC_FP32 && opts->refine_rtol > 0 &&
      (s = no_ard(prob, "iterative refinement")) != GP_OK)
    return s;
  if (opts->prec != GP_PREC_FP32 && opts->refine_rtol > 0)
    return refine_solve(prob, B, w, Xsol, nullptr, opts, iters, relres, ws, ws_bytes, st);
  const int kmax = precond_kmax(prob, opts->precond_rank);
  const size_t base = solve_bytes(prob, w, opts->prec);
  if (kmax > 0 && (s = check_ws(ws, ws_bytes, gp_workspace_bytes(GP_OP_PCG, prob, w, opts))) != GP_OK)
    return s;
  SolveSetup ss;
  if ((s = setup_solve(prob, w, false, opts->prec, 0, opts->prec, ws, ws_bytes, st, ss)) != GP_OK)
    return s;
  Precond pcond;
  if (kmax > 0) {
    pcond = carve_precond(static_cast<char*>(ws) + align256(base), ss.pc.nr_pad, prob->d, kmax,
                          ss.pc.w_pad);
    set_live_width(pcond, w);
    if ((s = build_precond(prob, kmax, opts->precond_tol, pcond, st)) != GP_OK) return s;
  }
  GP_CUDA(launch_pad_block(B, prob->n, w, w, ss.W.B, ss.pc.nr_pad, ss.pc.w_pad, 0, st));
  const int maxit = effective_maxit(prob, opts);
  s = run_cg(prob, ss.pc, opts->prec, ss.W, w, maxit, opts->cg_rtol, st, kmax > 0 ? &pcond : nullptr);
  if (s != GP_OK) return s;
  GP_CUDA(launch_unpad_block(ss.W.X, prob->n, w, ss.pc.w_pad, Xsol, w, 0, st));
  HostCg h;
  if ((s = read_cg(ss.W.S, h, st)) != GP_OK) return s;
  for (int c = 0; c < w; ++c) {
    if (iters) iters[c] = h.iters[c];
    if (relres) relres[c] = h.relres[c];
  }
  return check_conv(ss.W.S, w, maxit, opts->cg_rtol, st);
}

gp_status gp_pcg_solve_refined(const gp_problem* prob, const float* B, int32_t w, double* X64,
                               const gp_solve_opts* opts, int32_t* iters, double* relres, void* ws,
                               size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_width(w)) != GP_OK) return s;
  if ((s = check_opts(opts, false, true)) != GP_OK) return s;
  if (B == nullptr || X64 == nullptr) return fail(GP_ERR_ARG, "B and X64 must be non-NULL");
  if (!(opts->refine_rtol > 0)) return fail(GP_ERR_ARG, "refine_rtol must be > 0");
  if ((s = no_ard(prob, "iterative refinement")) != GP_OK) return s;
  return refine_solve(prob, B, w, nullptr, X64, opts, iters, relres, ws, ws_bytes,
                      static_cast<cudaStream_t>(stream));
}

gp_status gp_nystrom_apply(const gp_problem* prob, int32_t k, double tol, const float* V, int32_t w,
                           float* Z, float* L, int64_t* piv, int32_t* rank, void* ws,
                           size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_width(w)) != GP_OK) return s;
  if (k < 1 || k > GP_MAX_PRECOND_RANK) return fail(GP_ERR_ARG, "k must be in [1, 4096]");
  if (!(tol <= 1.0) && !(tol > 1.0)) return fail(GP_ERR_ARG, "tol is NaN");
  if (V == nullptr || Z == nullptr || rank == nullptr)
    return fail(GP_ERR_ARG, "V, Z and rank must be non-NULL");
  const int kmax = precond_kmax(prob, k);
  if ((s = check_ws(ws, ws_bytes, nystrom_entry_bytes(prob, w, kmax))) != GP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = prob->n;
  const int64_t n_pad = round_up(n, kPad);
  const int w_pad = static_cast<int>(round_up(w, 4));
  float* Vp = static_cast<float*>(ws);
  Precond pc = carve_precond(static_cast<char*>(ws) +
                                 align256(sizeof(float) * static_cast<size_t>(n_pad) * w_pad),
                             n_pad, prob->d, kmax, w_pad);
  GP_CUDA(cudaMemsetAsync(Vp, 0, sizeof(float) * static_cast<size_t>(n_pad) * w_pad, st));
  GP_CUDA(launch_pad_block(V, n, w, w, Vp, n_pad, w_pad, 0, st));
  if ((s = build_precond(prob, kmax, tol, pc, st)) != GP_OK) return s;
  GP_CUDA(nys_apply(pc.ws, pc.rank, n, pc.s, Vp, pc.Z, nullptr, st));
  GP_CUDA(launch_unpad_block(pc.Z, n, w, w_pad, Z, w, 0, st));
  if (L != nullptr)
    GP_CUDA(cudaMemcpy2DAsync(L, sizeof(float) * n, pc.ws.Lt, sizeof(float) * n_pad, sizeof(float) * n,
                              pc.rank, cudaMemcpyDeviceToDevice, st));
  if (piv != nullptr)
    GP_CUDA(cudaMemcpyAsync(piv, pc.ws.piv, sizeof(int64_t) * pc.rank, cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  *rank = pc.rank;
  return GP_OK;
}

gp_status gp_true_residual(const gp_problem* prob, const float* B, const float* X, int32_t w,
                           double* relres, void* ws, size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_width(w)) != GP_OK) return s;
  if (B == nullptr || X == nullptr || relres == nullptr)
    return fail(GP_ERR_ARG, "B, X and relres must be non-NULL");
  if ((s = no_ard(prob, "gp_true_residual")) != GP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = prob->n;
  const int64_t n_pad = round_up(n, kPad);
  const int w_pad = static_cast<int>(round_up(w, 4));
  if ((s = check_ws(ws, ws_bytes, carve_residual(nullptr, n, w).bytes)) != GP_OK) return s;
  const ResidualWs R = carve_residual(ws, n, w);
  const size_t plane = static_cast<size_t>(n_pad) * w_pad;
  // x64 = X over the padded plane (zero padding); the residual plane is fully
  // written by the combine (zero outside rows < n, columns < w).
  GP_CUDA(cudaMemsetAsync(R.x64, 0, plane * sizeof(double), st));
  GP_CUDA(cudaMemsetAsync(R.Bp, 0, plane * sizeof(float), st));
  GP_CUDA(cudaMemsetAsync(R.Xp, 0, plane * sizeof(float), st));
  GP_CUDA(cudaMemsetAsync(R.S, 0, sizeof(CgState), st));
  GP_CUDA(launch_pad_block(B, n, w, w, R.Bp, n_pad, w_pad, 0, st));
  GP_CUDA(launch_pad_block(X, n, w, w, R.Xp, n_pad, w_pad, 0, st));
  GP_CUDA(launch_refine_update(R.x64, R.Xp, n_pad, w_pad, w, st));   // x64 = X
  if ((s = residual_into(prob, R.Bp, w_pad, R.x64, w_pad, w, nullptr, n, kResF64, R.part, R.err,
                         R.r64, w_pad, nullptr, st)) != GP_OK)
    return s;
  GP_CUDA(launch_refine_norms(R.S, R.r64, R.Bp, R.rf, n_pad, w_pad, w, R.red, st));
  HostCg h;
  if ((s = read_cg(R.S, h, st)) != GP_OK) return s;
  for (int c = 0; c < w; ++c) relres[c] = h.relres[c];
  return GP_OK;
}

gp_status gp_residual_rows(const gp_problem* prob, const float* B, const double* X64, int32_t w,
                           const int64_t* rows, int64_t m, int32_t arith, double* R,
                           double* relres, void* ws, size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_width(w)) != GP_OK) return s;
  if (B == nullptr || X64 == nullptr) return fail(GP_ERR_ARG, "B and X64 must be non-NULL");
  if (m < 1 || m > prob->n) return fail(GP_ERR_ARG, "m must be in [1, n]");
  if (arith != GP_RESIDUAL_PAIR && arith != GP_RESIDUAL_FP64)
    return fail(GP_ERR_ARG, "arith must be GP_RESIDUAL_PAIR or GP_RESIDUAL_FP64");
  if (R == nullptr && relres == nullptr) return fail(GP_ERR_ARG, "R and relres are both NULL");
  if ((s = no_ard(prob, "gp_residual_rows")) != GP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = prob->n;
  if ((s = check_ws(ws, ws_bytes, carve_residual(nullptr, n, w).bytes)) != GP_OK) return s;
  const ResidualWs W = carve_residual(ws, n, w);
  const int64_t m_pad = round_up(m, kPad);
  const int w_pad = static_cast<int>(round_up(w, 4));
  // The residual rows land in the r64 plane, the B rows in Bp ([m_pad][w_pad],
  // zero padding written by the combine).
  if ((s = residual_into(prob, B, w, X64, w, w, rows, m, residual_arith(arith), W.part, W.err,
                         W.r64, w_pad, W.Bp, st)) != GP_OK)
    return s;
  int herr = 0;
  GP_CUDA(cudaMemcpyAsync(&herr, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (relres != nullptr) {
    GP_CUDA(cudaMemsetAsync(W.S, 0, sizeof(CgState), st));
    GP_CUDA(launch_refine_norms(W.S, W.r64, W.Bp, W.rf, m_pad, w_pad, w, W.red, st));
    HostCg h;
    if ((s = read_cg(W.S, h, st)) != GP_OK) return s;
    if (herr != 0) return fail(GP_ERR_ARG, "a row index is outside [0, n)");
    for (int c = 0; c < w; ++c) relres[c] = h.relres[c];
  }
  if (R != nullptr)
    GP_CUDA(cudaMemcpy2DAsync(R, sizeof(double) * w, W.r64, sizeof(double) * w_pad,
                              sizeof(double) * w, m, cudaMemcpyDeviceToDevice, st));
  GP_CUDA(cudaStreamSynchronize(st));
  if (herr != 0) return fail(GP_ERR_ARG, "a row index is outside [0, n)");
  return GP_OK;
}

gp_status gp_slq_logdet(const gp_problem* prob, const gp_solve_opts* opts, double* logdet,
                        double* logdet_stderr, void* ws, size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_opts(opts, true)) != GP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int p = opts->nprobe;
  SolveSetup ss;
  if ((s = setup_solve(prob, p, false, opts->prec, opts->nlanczos, slq_prec_of(opts), ws, ws_bytes,
                       st, ss)) != GP_OK)
    return s;
  if ((s = fill_probes(prob, opts, ss.W.B, ss.pc.nr_pad, ss.pc.w_pad, 0, st)) != GP_OK) return s;
  if ((s = run_lanczos(prob, ss.pl, ss.slq_prec, ss.W, 0, p, opts->nlanczos, st)) != GP_OK) return s;
  double out[16];
  GP_CUDA(cudaMemcpyAsync(out, ss.W.S2->out, sizeof(out), cudaMemcpyDeviceToHost, st));
  if ((s = device_status(&ss.W.S2->err, st)) != GP_OK) return s;
  if (logdet) *logdet = out[0];
  if (logdet_stderr) *logdet_stderr = out[1];
  return GP_OK;
}

// Gradient outputs of a backward pass: grad[3] (s, f, l), or grad[2 + d]
// (s, f, l_1..l_d) with per-dimension length-scales, whose info->quad/trace
// hold s and f in [0..1] and NaN in [2] (and no standard errors).
static gp_status write_grad(const gp_problem* prob, const SolveSetup& ss, const double out[16],
                            double* grad, gp_loss_info* info, cudaStream_t st) {
  if (!ss.kc.ard) {
    if (grad)
      for (int t = 0; t < 3; ++t) grad[t] = out[3 + t];
    if (info != nullptr)
      for (int t = 0; t < 3; ++t) {
        info->quad[t] = out[6 + t];
        info->trace[t] = out[9 + t];
        info->trace_stderr[t] = out[12 + t];
      }
    return GP_OK;
  }
  double g[2 + GP_MAX_DIM], q[2 + GP_MAX_DIM], tr[2 + GP_MAX_DIM];
  GP_CUDA(cudaMemcpyAsync(g, ss.W.S->ard_grad, sizeof(g), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaMemcpyAsync(q, ss.W.S->ard_quad, sizeof(q), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaMemcpyAsync(tr, ss.W.S->ard_trace, sizeof(tr), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  if (grad)
    for (int t = 0; t < 2 + prob->d; ++t) grad[t] = g[t];
  if (info != nullptr) {
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (int t = 0; t < 3; ++t) {
      info->quad[t] = t < 2 ? q[t] : nan;
      info->trace[t] = t < 2 ? tr[t] : nan;
      info->trace_stderr[t] = nan;
    }
  }
  return GP_OK;
}

gp_status gp_loss_and_grad(const gp_problem* prob, const float* y, const gp_solve_opts* opts,
                           double* loss, double* grad, gp_loss_info* info, void* ws, size_t ws_bytes,
                           void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_opts(opts, false, true)) != GP_OK) return s;
  if (opts->precond_rank > 0 && (s = no_ard(prob, "the preconditioned loss")) != GP_OK) return s;
  if (y == nullptr) return fail(GP_ERR_ARG, "y is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolveSetup ss;
  gp_status cgs = GP_OK;
  if ((s = forward_impl(prob, y, opts, true, ws, ws_bytes, st, ss, cgs)) != GP_OK) return s;
  if ((s = backward_impl(prob, opts, ss, st)) != GP_OK) return s;
  double out[16];
  if ((s = read_outputs(ss.W.S, opts->nprobe > 0 ? ss.W.S2 : nullptr, 1 + opts->nprobe, out, info,
                        st)) != GP_OK)
    return s;
  if (loss) *loss = out[2];
  if ((s = write_grad(prob, ss, out, grad, info, st)) != GP_OK) return s;
  return check_conv(ss.W.S, 1 + opts->nprobe, effective_maxit(prob, opts), opts->cg_rtol, st);
}

gp_status gp_loss_and_grad_batch(int32_t count, const gp_problem* probs, const float* const* y,
                                 const gp_solve_opts* opts, double* loss, double* grad,
                                 gp_loss_info* info, int32_t* status, void* const* ws,
                                 const size_t* ws_bytes, void* stream) {
  return loss_and_grad_batch(count, probs, y, opts, loss, grad, info, status, ws, ws_bytes,
                             static_cast<cudaStream_t>(stream));
}

gp_status gp_nll_forward(const gp_problem* prob, const float* y, const gp_solve_opts* opts, float* W,
                         double* loss, gp_loss_info* info, void* ws, size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_opts(opts, false)) != GP_OK) return s;
  if (y == nullptr || W == nullptr) return fail(GP_ERR_ARG, "y and W must be non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolveSetup ss;
  gp_status cgs = GP_OK;
  if ((s = forward_impl(prob, y, opts, true, ws, ws_bytes, st, ss, cgs)) != GP_OK) return s;
  const int w = 1 + opts->nprobe;
  GP_CUDA(launch_unpad_block(ss.W.X, prob->n, w, ss.pc.w_pad, W, w, 0, st));
  double out[16];
  if ((s = read_outputs(ss.W.S, opts->nprobe > 0 ? ss.W.S2 : nullptr, w, out, info, st)) != GP_OK)
    return s;
  if (loss) *loss = out[2];
  return check_conv(ss.W.S, w, effective_maxit(prob, opts), opts->cg_rtol, st);
}

gp_status gp_nll_backward(const gp_problem* prob, const gp_solve_opts* opts, const float* Wsol,
                          double* grad, gp_loss_info* info, void* ws, size_t ws_bytes,
                          void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_opts(opts, false)) != GP_OK) return s;
  if (Wsol == nullptr) return fail(GP_ERR_ARG, "W is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int w = 1 + opts->nprobe;
  SolveSetup ss;
  if ((s = setup_solve(prob, w, true, GP_PREC_FP32, 0, GP_PREC_FP32, ws, ws_bytes, st, ss)) != GP_OK)
    return s;
  // B = [alpha | Z] (alpha = column 0 of W), X = W.
  GP_CUDA(launch_pad_block(Wsol, prob->n, 1, w, ss.W.B, ss.pc.nr_pad, ss.pc.w_pad, 0, st));
  if ((s = fill_probes(prob, opts, ss.W.B, ss.pc.nr_pad, ss.pc.w_pad, 1, st)) != GP_OK) return s;
  GP_CUDA(cudaMemsetAsync(ss.W.X, 0, sizeof(float) * ss.pc.nr_pad * ss.pc.w_pad, st));
  GP_CUDA(launch_pad_block(Wsol, prob->n, w, w, ss.W.X, ss.pc.nr_pad, ss.pc.w_pad, 0, st));
  if ((s = backward_impl(prob, opts, ss, st)) != GP_OK) return s;
  double out[16];
  GP_CUDA(cudaMemcpyAsync(out, ss.W.S->out, sizeof(out), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  if ((s = write_grad(prob, ss, out, grad, info, st)) != GP_OK) return s;
  return device_status(&ss.W.S->err, st);
}

gp_status gp_predict_mean(const gp_problem* prob, const float* alpha, const float* Xstar, int64_t m,
                          float* mu, int32_t prec, void* ws, size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_prec(prec)) != GP_OK) return s;
  if (alpha == nullptr || Xstar == nullptr || mu == nullptr)
    return fail(GP_ERR_ARG, "alpha, Xstar and mu must be non-NULL");
  if (m < 1 || m > (int64_t(1) << 31) - 4096) return fail(GP_ERR_ARG, "m out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = prob->n;
  const SimtPlan p = plan_for(m, n, prob->d, 1, false, prob->kernel, GP_PREC_FP32);
  ProdWs L = carve_product(nullptr, p, false, true, GP_PREC_FP32);
  if ((s = check_ws(ws, ws_bytes, L.bytes)) != GP_OK) return s;
  L = carve_product(ws, p, false, true, GP_PREC_FP32);
  const KernelConsts kc = kernel_consts(prob);
  GP_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int), st));
  GP_CUDA(launch_stage_points(prob->X, n, prob->d, prob->d, prob->X, kc.csd, p.dp, p.nc_pad, L.xc, st));
  GP_CUDA(launch_stage_points(Xstar, m, prob->d, prob->d, prob->X, kc.csd, p.dp, p.nr_pad, L.xr, st));
  GP_CUDA(cudaMemsetAsync(L.vp, 0, sizeof(float) * p.nc_pad * p.w_pad, st));
  GP_CUDA(launch_pad_block(alpha, n, 1, 1, L.vp, p.nc_pad, p.w_pad, 0, st));
  if ((s = run_product(p, prob->kernel, false, GP_PREC_FP32, L.xr, L.xc, L.vp, nullptr, L.part_k, nullptr,
                       nullptr, L.err, st)) != GP_OK)
    return s;
  EpiArgs e{};
  e.part_k = L.part_k;
  e.split = p.split;
  e.nr_pad = p.nr_pad;
  e.w_pad = p.w_pad;
  e.n = m;
  e.w = 1;
  e.cK = prob->theta.f * prob->theta.f;
  e.y = mu;
  e.ldy = 1;
  e.err = L.err;
  GP_CUDA(launch_epilogue(e, st));
  return GP_OK;
}

gp_status gp_predict_var(const gp_problem* prob, const float* Xstar, int64_t m, float* var,
                         const gp_solve_opts* opts, int32_t* iters_max, double* relres_max,
                         void* ws, size_t ws_bytes, void* stream) {
  gp_status s;
  if ((s = check_problem(prob)) != GP_OK) return s;
  if ((s = check_opts(opts, false)) != GP_OK) return s;
  if (Xstar == nullptr || var == nullptr) return fail(GP_ERR_ARG, "Xstar and var must be non-NULL");
  if (m < 1 || m > (int64_t(1) << 31) - 4096) return fail(GP_ERR_ARG, "m out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = prob->n;
  const int prec = opts->prec;
  const int wb = static_cast<int>(std::min<int64_t>(m, GP_MAX_COLS));
  SolveSetup ss;
  if ((s = setup_solve(prob, wb, false, prec, 0, prec, ws, ws_bytes, st, ss)) != GP_OK) return s;
  const double f2 = prob->theta.f * prob->theta.f;
  const int maxit = effective_maxit(prob, opts);
  double inv_l[GP_MAX_DIM];
  for (int t = 0; t < prob->d; ++t) inv_l[t] = 1.0 / (prob->ls ? prob->ls[t] : prob->theta.l);
  int it_max = 0;
  double rel_max = 0.0;
  bool conv = true;
  // Test points in blocks of up to GP_MAX_COLS columns: B = f^2 K(X, X*_block),
  // U = Kh^-1 B by block CG, var = f^2 - diag(B^T U).
  for (int64_t c0 = 0; c0 < m; c0 += wb) {
    const int wl = static_cast<int>(std::min<int64_t>(wb, m - c0));
    GP_CUDA(cudaMemsetAsync(ss.W.S, 0, sizeof(CgState), st));
    GP_CUDA(cudaMemsetAsync(ss.W.S2, 0, sizeof(CgState), st));
    GP_CUDA(launch_cross_cols(prob->X, n, prob->d, Xstar + c0 * prob->d, wl, prob->kernel, inv_l,
                              f2, ss.W.B, ss.pc.nr_pad, ss.pc.w_pad, st));
    if ((s = run_cg(prob, ss.pc, prec, ss.W, wl, maxit, opts->cg_rtol, st)) != GP_OK) return s;
    GP_CUDA(launch_pred_var(ss.W.S2, ss.W.B, ss.W.X, ss.pc.nr_pad, ss.pc.w_pad, wl, f2, var + c0,
                            ss.W.red, st));
    HostCg h;
    if ((s = read_cg(ss.W.S, h, st)) != GP_OK) return s;
    for (int c = 0; c < wl; ++c) {
      it_max = std::max(it_max, h.iters[c]);
      rel_max = std::max(rel_max, h.relres[c]);
      conv = conv && !(h.relres[c] > opts->cg_rtol);
    }
  }
  if (iters_max) *iters_max = it_max;
  if (relres_max) *relres_max = rel_max;
  if (!conv) return fail(GP_ERR_NOT_CONVERGED, "predict_var: CG reached cg_maxit before cg_rtol");
  return GP_OK;
}

gp_status gp_profile_begin(void) {
  t_prof.on = true;
  t_prof.launches = 0;
  t_prof.product_launches = 0;
  t_prof.used = 0;
  return GP_OK;
}

gp_status gp_profile_end(double* product_ms, int64_t* product_launches, int64_t* total_launches) {
  double ms = 0.0;
  for (size_t i = 0; i < t_prof.used; ++i) {
    GP_CUDA(cudaEventSynchronize(t_prof.ev[i].second));
    float e = 0.f;
    GP_CUDA(cudaEventElapsedTime(&e, t_prof.ev[i].first, t_prof.ev[i].second));
    ms += e;
  }
  if (product_ms) *product_ms = ms;
  if (product_launches) *product_launches = t_prof.product_launches;
  if (total_launches) *total_launches = t_prof.launches;
  t_prof.on = false;
  t_prof.used = 0;
  return GP_OK;
}

gp_status gp_generate_probes(int64_t n, int32_t p, uint64_t seed, float* Z, int64_t ldz,
                             void* stream) {
  if (n < 1 || p < 1 || Z == nullptr || ldz < p) return fail(GP_ERR_ARG, "bad probe arguments");
  GP_CUDA(launch_probes(n, p, seed, Z, ldz, 0, n, static_cast<cudaStream_t>(stream)));
  return GP_OK;
}

}  // extern "C"
