// O(n w) kernels around the on-the-fly product: staging, epilogues, block CG
// (per-column CG with FP64 step scalars), probe generation, SLQ and the
// loss/gradient assembly.  All reductions are deterministic: per-block FP64
// partials in a fixed order, summed by the last block to finish (or, in the
// fused CG step, by every block after a grid barrier, in the same order).
#include <math.h>

#include <algorithm>

#include "tridiag.cuh"
#include "vec_kernels.cuh"

namespace gp {

namespace {

constexpr int kEltThreads = 256;

inline int elt_blocks(int64_t total) {
  int64_t b = (total + kEltThreads - 1) / kEltThreads;
  if (b > 152 * 32) b = 152 * 32;
  return static_cast<int>(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- reduction --
// Thread t of a block covers column c = t % w_pad and row lane t / w_pad.
struct RedLayout {
  int c, rl, nrl;
  bool live;
};

__device__ __forceinline__ RedLayout red_layout(int w_pad) {
  RedLayout L;
  L.nrl = kRedThreads / w_pad;
  L.c = threadIdx.x % w_pad;
  L.rl = threadIdx.x / w_pad;
  L.live = L.rl < L.nrl;
  return L;
}

__device__ __forceinline__ void block_rows(int64_t n_rows, int64_t& r0, int64_t& r1) {
  const int64_t per = (n_rows + gridDim.x - 1) / gridDim.x;
  r0 = static_cast<int64_t>(blockIdx.x) * per;
  r1 = r0 + per < n_rows ? r0 + per : n_rows;
}

// Combine the per-thread partials of NQ quantities into red[q][block][c].
template <int NQ>
__device__ __forceinline__ void block_store(const double (&acc)[NQ], const RedLayout& L, int w_pad,
                                            double* red) {
  __shared__ double sm[kRedThreads];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    sm[threadIdx.x] = L.live ? acc[q] : 0.0;
    __syncthreads();
    if (threadIdx.x < w_pad) {
      double s = 0.0;
      for (int k = 0; k < L.nrl; ++k) s += sm[k * w_pad + threadIdx.x];
      red[(static_cast<int64_t>(q) * gridDim.x + blockIdx.x) * w_pad + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// True in exactly one block: the last one to arrive (its reads of red see all).
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
    if (am_last) *ticket = 0u;
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

__device__ __forceinline__ double final_sum(const double* red, int q, int c, int w_pad) {
  double s = 0.0;
  for (int b = 0; b < static_cast<int>(gridDim.x); ++b)
    s += red[(static_cast<int64_t>(q) * gridDim.x + b) * w_pad + c];
  return s;
}

// Called by every thread of a block that has seen all partials (the last block
// to finish, or any block after a grid barrier): the sums over the grid's blocks of
// red[q][b][c] for q < nq (<= 3), c < w_pad, into shared memory (index
// q * w_pad + c).  With np = nq * w_pad pairs, lane l of the blockDim / np lanes
// of a pair adds blocks l, l + lanes, ...; the lanes are then added in lane
// order, so the result depends only on the launch shape, and the serial chain
// per thread is about gridDim / lanes loads instead of gridDim.
__device__ const double* final_sums(const double* red, int nq, int w_pad) {
  __shared__ double tot[3 * kMaxW];
  __shared__ double part[kRedThreads];
  const int np = nq * w_pad;
  const int t = threadIdx.x;
  const int nb = static_cast<int>(gridDim.x);
  const int nl = static_cast<int>(blockDim.x) / np;
  if (nl >= 1) {
    const int pr = t % np, l = t / np;
    double s = 0.0;
    if (l < nl) {
      const int q = pr / w_pad, c = pr - q * w_pad;
      for (int b = l; b < nb; b += nl) s += red[(static_cast<int64_t>(q) * nb + b) * w_pad + c];
    }
    part[t] = s;
    __syncthreads();
    if (t < np) {
      double a = 0.0;
      for (int k = 0; k < nl; ++k) a += part[k * np + t];
      tot[t] = a;
    }
  } else {
    for (int pr = t; pr < np; pr += blockDim.x) tot[pr] = final_sum(red, pr / w_pad, pr % w_pad, w_pad);
  }
  __syncthreads();
  return tot;
}

// ------------------------------------------------------------------ staging --

// Writes the staged layout of pt_index in order: element e is coordinate
// t = (e / 32) % dp of point i = (e / (32 dp)) * 32 + e % 32.
struct DimScales {
  float v[GP_MAX_DIM];
};

__global__ void stage_points_kernel(const float* X, int64_t n, int d, int64_t ld, const float* ref,
                                    DimScales cs, int dp, int64_t n_pad, float* out) {
  const int64_t total = n_pad * dp;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t tile = e / (32 * dp);
    const int rem = static_cast<int>(e - tile * 32 * dp);
    const int t = rem >> 5;
    const int64_t i = tile * 32 + (rem & 31);
    float v = 0.f;
    if (i < n && t < d) v = (X[i * ld + t] - ref[t]) * cs.v[t];
    out[e] = v;
  }
}

__global__ void pad_block_kernel(const float* V, int64_t n, int w, int64_t ldv, float* out,
                                 int64_t n_pad, int w_pad, int col_off) {
  const int64_t total = n_pad * w;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / w;
    const int c = static_cast<int>(e - i * w);
    out[i * w_pad + col_off + c] = (i < n) ? V[i * ldv + c] : 0.f;
  }
}

__global__ void unpad_block_kernel(const float* in, int64_t n, int w, int w_pad, float* out,
                                   int64_t ldo, int col_off) {
  const int64_t total = n * w;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / w;
    const int c = static_cast<int>(e - i * w);
    out[i * ldo + c] = in[i * w_pad + col_off + c];
  }
}

// SplitMix64 finaliser of (key + golden gamma): the first output of SplitMix64
// started from state `key` (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_first(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void probes_kernel(int64_t n, int p, uint64_t seed, float* Z, int64_t ldz, int col_off) {
  const int64_t total = n * p;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / p;
    const int c = static_cast<int>(e - i * p);
    const uint64_t key = seed ^ (static_cast<uint64_t>(c) << 40) ^ static_cast<uint64_t>(i);
    Z[i * ldz + col_off + c] = (splitmix64_first(key) >> 63) ? -1.f : 1.f;
  }
}

// ----------------------------------------------------------------- epilogue --

// Fixed-order compensated sum of the split partials of four adjacent columns:
// Knuth's two-sum carries each addition's rounding error in c, so the result is
// the exactly rounded sum up to a few units of FP32 rounding for any split count.
__device__ __forceinline__ float4 split_sum4(const float* part, int split, int64_t plane,
                                             int64_t idx) {
  float4 s = *reinterpret_cast<const float4*>(part + idx);
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
  auto two_sum = [](float& sv, float& cv, float p) {
    const float t = sv + p;
    const float bp = t - sv;
    cv += (sv - (t - bp)) + (p - bp);
    sv = t;
  };
  for (int k = 1; k < split; ++k) {
    const float4 p = *reinterpret_cast<const float4*>(part + k * plane + idx);
    two_sum(s.x, c.x, p.x);
    two_sum(s.y, c.y, p.y);
    two_sum(s.z, c.z, p.z);
    two_sum(s.w, c.w, p.w);
  }
  return make_float4(s.x + c.x, s.y + c.y, s.z + c.z, s.w + c.w);
}

// One thread per (row, four columns); w_pad is a multiple of 4, so the partial
// planes and V are read as float4 rows.
__global__ void epilogue_kernel(EpiArgs a) {
  const bool bad = (a.err != nullptr) && (*a.err != 0);
  const int nq = a.w_pad >> 2;
  const int64_t total = a.n * nq;
  const float qnan = __int_as_float(0x7fc00000);
  const int64_t plane = a.nr_pad * a.w_pad;
  const float cK = static_cast<float>(a.cK), cV = static_cast<float>(a.cV);
  const float cF = static_cast<float>(a.cF), cL = static_cast<float>(a.cL);
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / nq;
    const int c0 = static_cast<int>(e - i * nq) * 4;
    if (c0 >= a.w) continue;
    const int64_t idx = i * a.w_pad + c0;
    const float4 sk = split_sum4(a.part_k, a.split, plane, idx);
    float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.dyl != nullptr) sd = split_sum4(a.part_d, a.split, plane, idx);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.y != nullptr && a.cV != 0.0) v = *reinterpret_cast<const float4*>(a.v + idx);
    const float skv[4] = {sk.x, sk.y, sk.z, sk.w};
    const float sdv[4] = {sd.x, sd.y, sd.z, sd.w};
    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      if (c >= a.w) break;
      if (a.y != nullptr) a.y[i * a.ldy + c] = bad ? qnan : fmaf(cK, skv[u], cV * vv[u]);
      if (a.dyf != nullptr) a.dyf[i * a.ldf + c] = bad ? qnan : cF * skv[u];
      if (a.dyl != nullptr) a.dyl[i * a.ldl + c] = bad ? qnan : cL * sdv[u];
    }
  }
}

// ----------------------------------------------------------------- block CG --

__global__ void cg_init_kernel(CgState* S, const float* B, float* X, float* R, float* P,
                               int64_t n_pad, int w_pad, int w, int maxit, double rtol,
                               double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      const float b = B[idx];
      X[idx] = 0.f;
      R[idx] = b;
      P[idx] = b;
      acc[0] += static_cast<double>(b) * b;
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if (threadIdx.x < kMaxW) {
    const int c = threadIdx.x;
    double bn2 = 0.0;
    if (c < w_pad) bn2 = tot[c];
    const bool act = (c < w) && (bn2 > 0.0);
    S->bn2[c] = bn2;
    S->rr[c] = bn2;
    S->active[c] = act ? 1 : 0;
    S->iters[c] = 0;
    S->alpha[c] = 0.0;
    S->beta[c] = 0.0;
    S->relres[c] = act ? 1.0 : 0.0;
    if (act) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S->n_active = cnt;
    S->err = 0;
    S->iter = 0;
    S->bar_count = 0u;
    S->maxit = maxit;
    S->w = w;
    S->rtol = rtol;
  }
}

__global__ void cg_epi_alpha_kernel(CgState* S, const float* part_k, int split, const float* P,
                                    float* Q, int64_t n_pad, int64_t n, int w_pad, double f2,
                                    double snoise, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  const int64_t plane = n_pad * w_pad;
  double acc[1] = {0.0};
  if (L.live) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      float q = 0.f;
      if (r < n) {
        double sk = 0.0;
#pragma unroll 4
        for (int s = 0; s < split; ++s) sk += part_k[s * plane + idx];
        const double pv = P[idx];
        const double qd = f2 * sk + snoise * pv;
        q = static_cast<float>(qd);
        acc[0] += pv * static_cast<double>(q);
      }
      Q[idx] = q;
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    const double pap = tot[c];
    double al = 0.0;
    if (S->active[c]) {
      if (!(pap > 0.0) || !isfinite(pap)) {
        S->err = kDevBreakdown;
        S->active[c] = 0;
      } else {
        al = S->rr[c] / pap;
        const int it = S->iters[c];
        if (it < kMaxK) S->ahist[it][c] = al;
      }
    }
    S->alpha[c] = al;
  }
}

__global__ void cg_update_kernel(CgState* S, float* X, float* R, const float* P, const float* Q,
                                 int64_t n_pad, int w_pad, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live) {
    const int act = S->active[L.c];
    const float al = static_cast<float>(S->alpha[L.c]);
    if (act) {
      for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
        const int64_t idx = r * w_pad + L.c;
        X[idx] = fmaf(al, P[idx], X[idx]);
        const float rn = fmaf(-al, Q[idx], R[idx]);
        R[idx] = rn;
        acc[0] += static_cast<double>(rn) * rn;
      }
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    if (S->active[c]) {
      const double rr_new = tot[c];
      const double be = rr_new / S->rr[c];
      const int it = S->iters[c];
      if (it < kMaxK) S->bhist[it][c] = be;
      S->iters[c] = it + 1;
      S->rr[c] = rr_new;
      S->beta[c] = be;
      const double rel = sqrt(rr_new / S->bn2[c]);
      S->relres[c] = rel;
      if (!(rel > S->rtol) || it + 1 >= S->maxit || !isfinite(rel)) {
        S->active[c] = 0;
      } else {
        atomicAdd(&cnt, 1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S->n_active = cnt;
    S->iter = S->iter + 1;
  }
}

// Preconditioned CG (z = M^-1 r): X += alpha P; R -= alpha Q; ||R||^2 gives the
// relative residual and the stop test.  The recurrence scalar r^T z and beta
// come from pcg_rz_kernel after the preconditioner has been applied.
__global__ void pcg_update_kernel(CgState* S, float* X, float* R, const float* P, const float* Q,
                                  int64_t n_pad, int w_pad, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live) {
    const int act = S->active[L.c];
    const float al = static_cast<float>(S->alpha[L.c]);
    if (act) {
      for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
        const int64_t idx = r * w_pad + L.c;
        X[idx] = fmaf(al, P[idx], X[idx]);
        const float rn = fmaf(-al, Q[idx], R[idx]);
        R[idx] = rn;
        acc[0] += static_cast<double>(rn) * rn;
      }
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    if (S->active[c]) {
      const int it = S->iters[c];
      S->iters[c] = it + 1;
      const double rel = sqrt(tot[c] / S->bn2[c]);
      S->relres[c] = rel;
      if (!(rel > S->rtol) || it + 1 >= S->maxit || !isfinite(rel)) {
        S->active[c] = 0;
      } else {
        atomicAdd(&cnt, 1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S->n_active = cnt;
    S->iter = S->iter + 1;
  }
}

// rz_c = R_c^T Z_c; beta_c = rz_c / (previous rz_c) (0 when `first`); the
// previous value is replaced (S->rr holds r^T z in preconditioned CG, the
// numerator of alpha).  A non-positive or non-finite rz is a breakdown.
__global__ void pcg_rz_kernel(CgState* S, const float* R, const float* Z, int64_t n_pad, int w_pad,
                              int first, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      acc[0] += static_cast<double>(R[idx]) * Z[idx];
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    double be = 0.0;
    if (S->active[c]) {
      const double rz = tot[c];
      if (!(rz > 0.0) || !isfinite(rz)) {
        S->err = kDevBreakdown;
        S->active[c] = 0;
      } else {
        be = first ? 0.0 : rz / S->rr[c];
        S->rr[c] = rz;
      }
    }
    S->beta[c] = be;
  }
}

__global__ void cg_pupdate_kernel(CgState* S, const float* R, float* P, int64_t n_pad, int w_pad) {
  if (S->n_active == 0) return;
  const int64_t total = n_pad * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % w_pad);
    if (S->active[c]) P[e] = fmaf(static_cast<float>(S->beta[c]), P[e], R[e]);
  }
}

// Grid-wide barrier for a cooperative launch.  Writes of the block before the
// call are visible to every block after it (fence before the arrival, fence
// after the release).  The wait is bounded by time and by iterations: on
// timeout the block records kDevTimeout and the caller returns.
constexpr unsigned long long kBarrierNs = 4000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_barrier(CgState* S) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &S->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(&S->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&S->bar_count, 0u);
      __threadfence();
      atomicAdd(&S->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      for (long long it = 0; *gen == g; ++it) {
        if (it >= 16 * kSpinLimit || global_ns() - t0 > kBarrierNs) {
          atomicExch(&S->err, static_cast<int>(kDevTimeout));
          good = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// One CG iteration after the product: phase A is cg_epi_alpha (Q and p^T q,
// reduced in plane 0 of red), phase B cg_update (x, r and r^T r in plane 1),
// phase C cg_pupdate.  Every block reads the column state once before the
// first barrier and then derives alpha, beta and the stopping decisions from
// the same sums in the same order as the separate kernels' last block; block 0
// alone writes them back.  A thread touches only the rows of its own block, so
// the vectors need no barrier, only the sums do.
__global__ void __launch_bounds__(kRedThreads, 4)
    cg_step_kernel(CgState* S, const float* part_k, int split, float* X, float* R, float* P,
                   float* Q, int64_t n_pad, int64_t n, int w_pad, double f2, double snoise,
                   double* red) {
  if (S->n_active == 0 || S->err == kDevTimeout) return;
  __shared__ int act_s[kMaxW];
  __shared__ int it_s[kMaxW];
  __shared__ double rr_s[kMaxW];
  __shared__ double coef_s[kMaxW];
  __shared__ int cnt;
  const bool writer = blockIdx.x == 0;
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    act_s[c] = S->active[c];
    it_s[c] = S->iters[c];
    rr_s[c] = S->rr[c];
  }
  if (threadIdx.x == 0) cnt = 0;
  const double rtol = S->rtol;
  const int maxit = S->maxit;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  const int64_t plane = n_pad * w_pad;
  double* red_b = red + static_cast<int64_t>(gridDim.x) * w_pad;

  // A: Q = f^2 sum_s partK + s P on live rows (0 on padding rows); p^T q.
  double acc[1] = {0.0};
  if (L.live) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      float q = 0.f;
      if (r < n) {
        double sk = 0.0;
#pragma unroll 4
        for (int s = 0; s < split; ++s) sk += part_k[s * plane + idx];
        const double pv = P[idx];
        const double qd = f2 * sk + snoise * pv;
        q = static_cast<float>(qd);
        acc[0] += pv * static_cast<double>(q);
      }
      Q[idx] = q;
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!grid_barrier(S)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    const double pap = tot[c];
    double al = 0.0;
    if (act_s[c]) {
      if (!(pap > 0.0) || !isfinite(pap)) {
        act_s[c] = 0;
        if (writer) {
          S->err = kDevBreakdown;
          S->active[c] = 0;
        }
      } else {
        al = rr_s[c] / pap;
        if (writer && it_s[c] < kMaxK) S->ahist[it_s[c]][c] = al;
      }
    }
    coef_s[c] = al;
    if (writer) S->alpha[c] = al;
  }
  __syncthreads();

  // B: x += alpha p; r -= alpha q; r^T r.
  acc[0] = 0.0;
  if (L.live && act_s[L.c]) {
    const float al = static_cast<float>(coef_s[L.c]);
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      X[idx] = fmaf(al, P[idx], X[idx]);
      const float rn = fmaf(-al, Q[idx], R[idx]);
      R[idx] = rn;
      acc[0] += static_cast<double>(rn) * rn;
    }
  }
  block_store<1>(acc, L, w_pad, red_b);
  if (!grid_barrier(S)) return;
  tot = final_sums(red_b, 1, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    double be = 0.0;
    if (act_s[c]) {
      const double rr_new = tot[c];
      be = rr_new / rr_s[c];
      const int it = it_s[c];
      const double rel = sqrt(rr_new / S->bn2[c]);
      const bool stop = !(rel > rtol) || it + 1 >= maxit || !isfinite(rel);
      if (writer) {
        if (it < kMaxK) S->bhist[it][c] = be;
        S->iters[c] = it + 1;
        S->rr[c] = rr_new;
        S->beta[c] = be;
        S->relres[c] = rel;
        if (stop) S->active[c] = 0;
      }
      if (stop)
        act_s[c] = 0;
      else
        atomicAdd(&cnt, 1);
    }
    coef_s[c] = be;
  }
  __syncthreads();
  if (writer && threadIdx.x == 0) {
    S->n_active = cnt;
    S->iter = S->iter + 1;
  }

  // C: p = r + beta p on the columns still iterating.
  if (L.live && act_s[L.c]) {
    const float be = static_cast<float>(coef_s[L.c]);
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      P[idx] = fmaf(be, P[idx], R[idx]);
    }
  }
}

// ------------------------------------------------------------------ Lanczos --
// One independent Lanczos process per active column, with full
// reorthogonalisation by two classical Gram-Schmidt passes per step, the steps
// of stochastic Lanczos quadrature (Ubaru et al. 2017) from q_0 = z/||z||.

// bn2 = ||B_c||^2, or B_c^T B2_c when B2 is given (preconditioned Lanczos:
// z^T M^-1 z with B2 = M^-1 B).
__global__ void lz_init_kernel(CgState* S, const float* B, const float* B2, int64_t n_pad, int w_pad,
                               int col0, int p, double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live)
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const double b = B[r * w_pad + L.c];
      acc[0] += b * (B2 != nullptr ? static_cast<double>(B2[r * w_pad + L.c]) : b);
    }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if (threadIdx.x < kMaxW) {
    const int c = threadIdx.x;
    const double bn2 = c < w_pad ? tot[c] : 0.0;
    const bool act = c >= col0 && c < col0 + p && bn2 > 0.0;
    S->bn2[c] = bn2;
    S->active[c] = act ? 1 : 0;
    S->iters[c] = 0;
    S->tnorm[c] = 0.0;
    S->alpha[c] = 0.0;
    S->beta[c] = 0.0;
    if (act) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S->n_active = cnt;
    S->err = 0;
    S->iter = 0;
  }
}

// dst = src * scale_c for active columns, 0 otherwise; scale = 1/sqrt(bn2) (j < 0)
// or 1/beta_j.
__global__ void lz_scale_kernel(const CgState* S, const float* src, float* dst, int64_t n_pad,
                                int w_pad, int j) {
  const int64_t total = n_pad * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % w_pad);
    float v = 0.f;
    if (S->active[c]) {
      const double sc = j < 0 ? 1.0 / sqrt(S->bn2[c]) : 1.0 / S->bhist[j][c];
      v = static_cast<float>(static_cast<double>(src[e]) * sc);
    }
    dst[e] = v;
  }
}

__global__ void lz_epi_alpha_kernel(CgState* S, const float* part_k, int split, const float* Qj,
                                    float* W, int64_t n_pad, int64_t n, int w_pad, double f2,
                                    double snoise, int j, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  const int64_t plane = n_pad * w_pad;
  double acc[1] = {0.0};
  if (L.live) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      float wv = 0.f;
      if (r < n) {
        double sk = 0.0;
#pragma unroll 4
        for (int s = 0; s < split; ++s) sk += part_k[s * plane + idx];
        const double qv = Qj[idx];
        wv = static_cast<float>(f2 * sk + snoise * qv);
        acc[0] += qv * static_cast<double>(wv);
      }
      W[idx] = wv;
    }
  }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    const double al = tot[c];
    if (S->active[c]) S->ahist[j][c] = al;
  }
}

__global__ void lz_three_term_kernel(const CgState* S, float* W, const float* Q, int64_t n_pad,
                                     int w_pad, int j) {
  if (S->n_active == 0) return;
  const int64_t plane = n_pad * w_pad;
  const float* Qj = Q + static_cast<int64_t>(j) * plane;
  const float* Qm = j > 0 ? Q + static_cast<int64_t>(j - 1) * plane : nullptr;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < plane;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % w_pad);
    if (!S->active[c]) continue;
    double v = static_cast<double>(W[e]) - S->ahist[j][c] * static_cast<double>(Qj[e]);
    if (j > 0) v -= S->bhist[j - 1][c] * static_cast<double>(Qm[e]);
    W[e] = static_cast<float>(v);
  }
}

// h[i][c] = sum_r Q_i[r][c] W[r][c] for i < nq.
__global__ void lz_dots_kernel(CgState* S, const float* W, const float* Q, int64_t n_pad, int w_pad,
                               int nq, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  const int64_t plane = n_pad * w_pad;
  // Eight basis vectors per pass: their loads are independent, so they are in
  // flight together instead of one round trip per basis vector; the block sums
  // of the eight are then formed by eight groups of threads at once.
  constexpr int kChunk = 8;
  __shared__ double sm[kChunk][kRedThreads];
  for (int i0 = 0; i0 < nq; i0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) acc[k] = 0.0;
    if (L.live) {
      for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
        const int64_t idx = r * w_pad + L.c;
        const double wv = static_cast<double>(W[idx]);
#pragma unroll
        for (int k = 0; k < kChunk; ++k)
          if (i0 + k < nq)
            acc[k] += static_cast<double>(Q[static_cast<int64_t>(i0 + k) * plane + idx]) * wv;
      }
    }
#pragma unroll
    for (int k = 0; k < kChunk; ++k) sm[k][threadIdx.x] = L.live ? acc[k] : 0.0;
    __syncthreads();
    const int nk = min(kChunk, nq - i0);
    for (int t = threadIdx.x; t < nk * w_pad; t += blockDim.x) {
      const int k = t / w_pad;
      const int c = t - k * w_pad;
      double sum = 0.0;
      for (int q = 0; q < L.nrl; ++q) sum += sm[k][q * w_pad + c];
      red[(static_cast<int64_t>(i0 + k) * gridDim.x + blockIdx.x) * w_pad + c] = sum;
    }
    __syncthreads();
  }
  if (!last_block(&S->ticket)) return;
  for (int t = threadIdx.x; t < nq * w_pad; t += blockDim.x) {
    const int i = t / w_pad;
    const int c = t - i * w_pad;
    S->h[i][c] = final_sum(red, i, c, w_pad);
  }
}

__global__ void lz_sub_kernel(const CgState* S, float* W, const float* Q, int64_t n_pad, int w_pad,
                              int nq) {
  if (S->n_active == 0) return;
  const int64_t plane = n_pad * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < plane;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % w_pad);
    if (!S->active[c]) continue;
    double v = W[e];
    for (int i = 0; i < nq; ++i) v -= S->h[i][c] * static_cast<double>(Q[i * plane + e]);
    W[e] = static_cast<float>(v);
  }
}

// beta_j = ||W|| per column, or sqrt(W^T W2) when W2 is given (the M-norm of
// the preconditioned Lanczos vector W with W2 = M W).
__global__ void lz_norm_kernel(CgState* S, const float* W, const float* W2, int64_t n_pad, int w_pad,
                               int j, int k, double* red) {
  if (S->n_active == 0) return;
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live)
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const double v = W[r * w_pad + L.c];
      acc[0] += v * (W2 != nullptr ? static_cast<double>(W2[r * w_pad + L.c]) : v);
    }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    if (S->active[c]) {
      const double be = sqrt(fmax(tot[c], 0.0));
      const double bprev = j > 0 ? S->bhist[j - 1][c] : 0.0;
      const double tn = fmax(S->tnorm[c], fabs(S->ahist[j][c]) + be + bprev);
      S->tnorm[c] = tn;
      S->bhist[j][c] = be;
      S->iters[c] = j + 1;
      if (j + 1 >= k || !(be >= 1e-14 * tn)) {
        S->active[c] = 0;
      } else {
        atomicAdd(&cnt, 1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) S->n_active = cnt;
}

// ---------------------------------------------------------------------- SLQ --

// One block per probe (thread 0 works: the QR sweeps of different probes take
// different paths, so they run in separate warps); the last block to finish
// forms the mean and standard error over the probes in probe order.
__global__ void slq_kernel(CgState* S, int col0, int p, int k) {
  const int i = blockIdx.x;
  if (threadIdx.x == 0) {
    const int c = col0 + i;
    int m = S->iters[c];
    if (m > k) m = k;
    // The QR sweeps' working arrays in shared memory (shorter latency than the
    // local-memory stack frame on their serial path).
    __shared__ double a[kMaxK], b[kMaxK], q[kMaxK];
    bool ok = true;
    const double v = lanczos_logquad(&S->ahist[0][c], &S->bhist[0][c], kMaxW, m, S->bn2[c], a, b,
                                     q, &ok);
    S->slq_val[i] = v;
    if (!ok) atomicExch(&S->err, kDevNumeric);
  }
  if (!last_block(&S->ticket)) return;
  if (threadIdx.x == 0) {
    double mean = 0.0;
    for (int j = 0; j < p; ++j) mean += S->slq_val[j];
    mean = p > 0 ? mean / p : 0.0;
    double var = 0.0;
    for (int j = 0; j < p; ++j) var += (S->slq_val[j] - mean) * (S->slq_val[j] - mean);
    const double se = p > 1 ? sqrt(var / (p - 1) / p) : 0.0;
    S->out[0] = mean;
    S->out[1] = se;
  }
}

// ------------------------------------------------------------ gradient pass --

__global__ void grad_dots_kernel(CgState* S, const float* part_k, const float* part_d, int split,
                                 const float* V, const float* W, int64_t n_pad, int w_pad, int w,
                                 double cF, double cL, double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  const int64_t plane = n_pad * w_pad;
  double acc[3] = {0.0, 0.0, 0.0};
  if (L.live && L.c < w) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      const double wv = W[idx];
      if (wv == 0.0) continue;
      double sk = 0.0, sd = 0.0;
      for (int s = 0; s < split; ++s) {
        sk += part_k[s * plane + idx];
        sd += part_d[s * plane + idx];
      }
      acc[0] += wv * static_cast<double>(V[idx]);
      acc[1] += wv * (cF * sk);
      acc[2] += wv * (cL * sd);
    }
  }
  block_store<3>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 3, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    for (int q = 0; q < 3; ++q) S->dots[q][c] = tot[q * w_pad + c];
  }
}

__global__ void yalpha_kernel(CgState* S, const float* B, const float* X, int64_t n_pad, int w_pad,
                              double* red) {
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
    acc[0] += static_cast<double>(B[r * w_pad]) * static_cast<double>(X[r * w_pad]);
  RedLayout L;
  L.nrl = kRedThreads;
  L.c = 0;
  L.rl = threadIdx.x;
  L.live = true;
  block_store<1>(acc, L, 1, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, 1);
  if (threadIdx.x == 0) S->yalpha = tot[0];
}

// out: [0] logdet [1] logdet_stderr [2] loss [3..5] grad [6..8] quad [9..11] trace
//      [12..14] trace_stderr [15] y^T alpha
__global__ void assemble_kernel(CgState* S, int64_t n, int p) {
  if (threadIdx.x != 0) return;
  const double log2pi = 1.8378770664093454835606594728112;
  const double ya = S->yalpha;
  const double logdet = S->out[0];
  S->out[2] = 0.5 * (ya + logdet + static_cast<double>(n) * log2pi);
  for (int t = 0; t < 3; ++t) {
    const double quad = S->dots[t][0];
    double mean = 0.0;
    for (int i = 1; i <= p; ++i) mean += S->dots[t][i];
    mean = p > 0 ? mean / p : 0.0;
    double var = 0.0;
    for (int i = 1; i <= p; ++i) var += (S->dots[t][i] - mean) * (S->dots[t][i] - mean);
    S->out[6 + t] = quad;
    mean += S->trm[t];   // tr(M^-1 dM/dtheta) of a preconditioner (0 for M = I)
    S->out[9 + t] = mean;
    S->out[12 + t] = p > 1 ? sqrt(var / (p - 1) / p) : 0.0;
    S->out[3 + t] = 0.5 * (-quad + mean);
  }
  S->out[15] = ya;
}

// out[c] = sum_r A[r][c] B[r][c] (FP64, fixed order) for every column c < w_pad.
__global__ void plane_dots_kernel(CgState* S, const float* A, const float* B, int64_t n_pad,
                                  int w_pad, double* out, double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live)
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      acc[0] += static_cast<double>(A[idx]) * static_cast<double>(B[idx]);
    }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w_pad) out[threadIdx.x] = tot[threadIdx.x];
}

// Eq. 2's Hutchinson terms with a preconditioner: for probe columns c in
// [1, 1 + p) with v = M^-1 z_c, subtract v^T (dM/dtheta) v from the dots
// W_c^T dKh V_c: s: v^T v (S->vv); f: (2/f) ||L^T v||^2; l: 2 (L^T v).(dL^T v),
// with U = L^T V and U2 = (dL/dl)^T V ([r][w_pad], FP64).
__global__ void precond_corr_kernel(CgState* S, const double* U, const double* U2, int r, int w_pad,
                                    int p, double f) {
  const int c = 1 + static_cast<int>(threadIdx.x);
  if (c > p) return;
  double uu = 0.0, ud = 0.0;
  for (int m = 0; m < r; ++m) {
    const double u = U[static_cast<int64_t>(m) * w_pad + c];
    uu += u * u;
    ud += u * U2[static_cast<int64_t>(m) * w_pad + c];
  }
  S->dots[0][c] -= S->vv[c];
  S->dots[1][c] -= (2.0 / f) * uu;
  S->dots[2][c] -= 2.0 * ud;
}

__global__ void add_logdet_m_kernel(CgState* S) {
  if (threadIdx.x == 0 && blockIdx.x == 0) S->out[0] += S->logdet_m;
}

__global__ void copy_col0_kernel(const float* X, float* V, int64_t n_pad, int w_pad) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n_pad;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    V[r * w_pad] = X[r * w_pad];
}

// ------------------------------------------------------------ refinement --
// Norms of the outer residual of iterative refinement, the FP64 solution update
// and its FP32 copy.  (The residual itself is in residual.cuh.)
__global__ void widen_kernel(const float* a, double* b, int64_t total) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    b[e] = static_cast<double>(a[e]);
}

__global__ void refine_norms_kernel(CgState* S, const double* r64, const float* B, float* rf,
                                    int64_t n_pad, int w_pad, int w, double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[2] = {0.0, 0.0};
  if (L.live) {
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      const double rv = L.c < w ? r64[idx] : 0.0;
      const double bv = L.c < w ? static_cast<double>(B[idx]) : 0.0;
      rf[idx] = static_cast<float>(rv);
      acc[0] += rv * rv;
      acc[1] += bv * bv;
    }
  }
  block_store<2>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 2, w_pad);
  if (threadIdx.x < w_pad) {
    const int c = threadIdx.x;
    const double rr = tot[c];
    const double bb = tot[w_pad + c];
    S->rr[c] = rr;
    S->bn2[c] = bb;
    S->relres[c] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

__global__ void refine_update_kernel(double* x64, const float* X, int64_t n_pad, int w_pad, int w) {
  const int64_t total = n_pad * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (static_cast<int>(e % w_pad) < w) x64[e] += static_cast<double>(X[e]);
}

__global__ void refine_out_kernel(const double* x64, float* Xsol, int64_t n, int w_pad, int w) {
  const int64_t total = n * w;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / w;
    const int c = static_cast<int>(e - i * w);
    Xsol[e] = static_cast<float>(x64[i * w_pad + c]);
  }
}

// ------------------------------------------------------------ prediction --
// The cross-covariance columns of the posterior variance: B[j][c] =
// f^2 k(rho(x_j, x*_c)) for j < n, c < w from the unscaled FP32 points
// (rho^2 = sum_t ((x_jt - x*_ct) / l_t)^2; CUDA's expf and sqrtf), zero
// elsewhere in the padded [n_pad][w_pad] block.
__global__ void cross_cols_kernel(const float* X, int64_t n, int d, const float* Xs, int w,
                                  int kernel, DimScales inv_l, float f2, float* B, int64_t n_pad,
                                  int w_pad) {
  const int64_t total = n_pad * w_pad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = e / w_pad;
    const int c = static_cast<int>(e - j * w_pad);
    float v = 0.0f;
    if (j < n && c < w) {
      float r2 = 0.0f;
      for (int t = 0; t < d; ++t) {
        const float df = (X[j * d + t] - Xs[static_cast<int64_t>(c) * d + t]) * inv_l.v[t];
        r2 = fmaf(df, df, r2);
      }
      if (kernel == GP_KERNEL_GAUSSIAN) {
        v = f2 * expf(-0.5f * r2);
      } else {
        const float a = 1.7320508075688772f * sqrtf(r2);
        v = f2 * (1.0f + a) * expf(-a);
      }
    }
    B[e] = v;
  }
}

// S->dots[0][c] = sum_i A[i][c] B[i][c] (FP64 sums, fixed order) for c < w.
__global__ void coldots_kernel(CgState* S, const float* A, const float* B, int64_t n_pad, int w_pad,
                               int w, double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live)
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      acc[0] += static_cast<double>(A[idx]) * static_cast<double>(B[idx]);
    }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w_pad) S->dots[0][threadIdx.x] = threadIdx.x < w ? tot[threadIdx.x] : 0.0;
}

// var[c] = f2 - sum_j B[j][c] U[j][c] (FP64 sums, fixed order) for c < w.
__global__ void pred_var_kernel(CgState* S, const float* B, const float* U, int64_t n_pad,
                                int w_pad, int w, double f2, float* var, double* red) {
  const RedLayout L = red_layout(w_pad);
  int64_t r0, r1;
  block_rows(n_pad, r0, r1);
  double acc[1] = {0.0};
  if (L.live)
    for (int64_t r = r0 + L.rl; r < r1; r += L.nrl) {
      const int64_t idx = r * w_pad + L.c;
      acc[0] += static_cast<double>(B[idx]) * static_cast<double>(U[idx]);
    }
  block_store<1>(acc, L, w_pad, red);
  if (!last_block(&S->ticket)) return;
  const double* tot = final_sums(red, 1, w_pad);
  if (threadIdx.x < w) var[threadIdx.x] = static_cast<float>(f2 - tot[threadIdx.x]);
}

}  // namespace

// Blocks of the reducing O(n w) kernels: about 32 rows per block (each thread a
// row or two: these kernels are latency-bound at small n), at most 4 per SM.
int red_blocks(int64_t n_pad) {
  int64_t b = n_pad / 32;
  if (b > 608) b = 608;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

cudaError_t launch_stage_points(const float* X, int64_t n, int d, int64_t ld, const float* ref,
                                const float* cs, int dp, int64_t n_pad, float* out, cudaStream_t st) {
  DimScales sc{};
  for (int t = 0; t < d && t < GP_MAX_DIM; ++t) sc.v[t] = cs[t];
  stage_points_kernel<<<elt_blocks(n_pad * dp), kEltThreads, 0, st>>>(X, n, d, ld, ref, sc, dp,
                                                                      n_pad, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pad_block(const float* V, int64_t n, int w, int64_t ldv, float* out,
                             int64_t n_pad, int w_pad, int col_off, cudaStream_t st) {
  pad_block_kernel<<<elt_blocks(n_pad * w), kEltThreads, 0, st>>>(V, n, w, ldv, out, n_pad, w_pad,
                                                                  col_off);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_unpad_block(const float* in, int64_t n, int w, int w_pad, float* out,
                               int64_t ldo, int col_off, cudaStream_t st) {
  unpad_block_kernel<<<elt_blocks(n * w), kEltThreads, 0, st>>>(in, n, w, w_pad, out, ldo, col_off);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_probes(int64_t n, int p, uint64_t seed, float* Z, int64_t ldz, int col_off,
                          int64_t, cudaStream_t st) {
  if (n <= 0 || p <= 0) return cudaSuccess;
  probes_kernel<<<elt_blocks(n * p), kEltThreads, 0, st>>>(n, p, seed, Z, ldz, col_off);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_epilogue(const EpiArgs& a, cudaStream_t st) {
  epilogue_kernel<<<elt_blocks(a.n * (a.w_pad / 4)), kEltThreads, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_init(CgState* S, const float* B, float* X, float* R, float* P, int64_t n_pad,
                           int w_pad, int w, int maxit, double rtol, double* red, cudaStream_t st) {
  cg_init_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, B, X, R, P, n_pad, w_pad, w, maxit,
                                                            rtol, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_epi_alpha(CgState* S, const float* part_k, int split, const float* P,
                                float* Q, int64_t n_pad, int64_t n, int w_pad, double f2,
                                double snoise, double* red, cudaStream_t st) {
  cg_epi_alpha_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, part_k, split, P, Q, n_pad, n,
                                                                 w_pad, f2, snoise, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_update(CgState* S, float* X, float* R, const float* P, const float* Q,
                             int64_t n_pad, int w_pad, double* red, cudaStream_t st) {
  cg_update_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, X, R, P, Q, n_pad, w_pad, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_pupdate(CgState* S, const float* R, float* P, int64_t n_pad, int w_pad,
                              cudaStream_t st) {
  cg_pupdate_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, R, P, n_pad, w_pad);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(CgState* S, float* X, float* R, const float* P, const float* Q,
                              int64_t n_pad, int w_pad, double* red, cudaStream_t st) {
  pcg_update_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, X, R, P, Q, n_pad, w_pad, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_rz(CgState* S, const float* R, const float* Z, int64_t n_pad, int w_pad,
                          bool first, double* red, cudaStream_t st) {
  pcg_rz_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, R, Z, n_pad, w_pad, first ? 1 : 0, red);
  count_launch();
  return cudaGetLastError();
}

bool cg_step_fits(int64_t n_pad) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_step_kernel, kRedThreads, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return coop != 0 && static_cast<int64_t>(red_blocks(n_pad)) <= static_cast<int64_t>(per_sm) * sms;
}

cudaError_t launch_cg_step(CgState* S, const float* part_k, int split, float* X, float* R, float* P,
                           float* Q, int64_t n_pad, int64_t n, int w_pad, double f2, double snoise,
                           double* red, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(red_blocks(n_pad));
  cfg.blockDim = dim3(kRedThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, cg_step_kernel, S, part_k, split, X, R, P, Q, n_pad,
                                           n, w_pad, f2, snoise, red);
  count_launch();
  return e;
}

cudaError_t launch_lz_init(CgState* S, const float* B, float* Q0, int64_t n_pad, int w_pad, int col0,
                           int p, double* red, cudaStream_t st) {
  lz_init_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, B, nullptr, n_pad, w_pad, col0, p, red);
  count_launch();
  lz_scale_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, B, Q0, n_pad, w_pad, -1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lz_epi_alpha(CgState* S, const float* part_k, int split, const float* Qj,
                                float* W, int64_t n_pad, int64_t n, int w_pad, double f2,
                                double snoise, int j, double* red, cudaStream_t st) {
  lz_epi_alpha_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, part_k, split, Qj, W, n_pad, n,
                                                                 w_pad, f2, snoise, j, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lz_three_term(CgState* S, float* W, const float* Q, int64_t n_pad, int w_pad,
                                 int j, cudaStream_t st) {
  lz_three_term_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, W, Q, n_pad, w_pad, j);
  count_launch();
  return cudaGetLastError();
}

int lz_dot_blocks(int64_t n_pad) { return std::min(red_blocks(n_pad), kLzDotBlocks); }

cudaError_t launch_lz_reorth(CgState* S, float* W, const float* Q, int64_t n_pad, int w_pad, int j,
                             double* red, cudaStream_t st) {
  lz_dots_kernel<<<lz_dot_blocks(n_pad), kRedThreads, 0, st>>>(S, W, Q, n_pad, w_pad, j + 1, red);
  count_launch();
  lz_sub_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, W, Q, n_pad, w_pad, j + 1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lz_norm_next(CgState* S, const float* W, float* Q, int64_t n_pad, int w_pad,
                                int j, int k, double* red, cudaStream_t st) {
  lz_norm_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, W, nullptr, n_pad, w_pad, j, k, red);
  count_launch();
  if (j + 1 < k) {
    float* Qn = Q + static_cast<int64_t>(j + 1) * n_pad * w_pad;
    lz_scale_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, W, Qn, n_pad, w_pad, j);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_lz_init_m(CgState* S, const float* Z, const float* V, float* Q0, float* P0,
                             int64_t n_pad, int w_pad, int col0, int p, double* red, cudaStream_t st) {
  lz_init_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, Z, V, n_pad, w_pad, col0, p, red);
  count_launch();
  lz_scale_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, V, Q0, n_pad, w_pad, -1);
  count_launch();
  lz_scale_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, Z, P0, n_pad, w_pad, -1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lz_reorth_m(CgState* S, float* U, float* MU, const float* Q, const float* P,
                               int64_t n_pad, int w_pad, int j, double* red, cudaStream_t st) {
  lz_dots_kernel<<<lz_dot_blocks(n_pad), kRedThreads, 0, st>>>(S, U, P, n_pad, w_pad, j + 1, red);
  count_launch();
  lz_sub_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, U, Q, n_pad, w_pad, j + 1);
  count_launch();
  lz_sub_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, MU, P, n_pad, w_pad, j + 1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lz_mnorm_next(CgState* S, const float* U, const float* MU, float* Q, float* P,
                                 int64_t n_pad, int w_pad, int j, int k, double* red, cudaStream_t st) {
  lz_norm_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, U, MU, n_pad, w_pad, j, k, red);
  count_launch();
  if (j + 1 < k) {
    const int64_t off = static_cast<int64_t>(j + 1) * n_pad * w_pad;
    lz_scale_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, U, Q + off, n_pad, w_pad, j);
    count_launch();
    lz_scale_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(S, MU, P + off, n_pad, w_pad, j);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_plane_dots(CgState* S, const float* A, const float* B, int64_t n_pad, int w_pad,
                              double* out, double* red, cudaStream_t st) {
  plane_dots_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, A, B, n_pad, w_pad, out, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_precond_corr(CgState* S, const double* U, const double* U2, int r, int w_pad, int p,
                                double f, cudaStream_t st) {
  precond_corr_kernel<<<1, kMaxW, 0, st>>>(S, U, U2, r, w_pad, p, f);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_add_logdet_m(CgState* S, cudaStream_t st) {
  add_logdet_m_kernel<<<1, 32, 0, st>>>(S);
  count_launch();
  return cudaGetLastError();
}

size_t red_doubles(int64_t n_pad, int w_pad) {
  const size_t a = 3 * static_cast<size_t>(red_blocks(n_pad));
  const size_t b = static_cast<size_t>(kMaxK + 1) * lz_dot_blocks(n_pad);
  return std::max(a, b) * w_pad;
}

cudaError_t launch_slq(CgState* S, int col0, int p, int k, cudaStream_t st) {
  if (p < 1) return cudaSuccess;
  slq_kernel<<<p, 32, 0, st>>>(S, col0, p, k);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_grad_dots(CgState* S, const float* part_k, const float* part_d, int split,
                             const float* V, const float* W, int64_t n_pad, int w_pad, int w,
                             double cF, double cL, double* red, cudaStream_t st) {
  grad_dots_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, part_k, part_d, split, V, W, n_pad,
                                                              w_pad, w, cF, cL, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_yalpha(CgState* S, const float* B, const float* X, int64_t n_pad, int w_pad,
                          double* red, cudaStream_t st) {
  yalpha_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, B, X, n_pad, w_pad, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_assemble(CgState* S, int64_t n, int p, cudaStream_t st) {
  assemble_kernel<<<1, 32, 0, st>>>(S, n, p);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* a, double* b, int64_t total, cudaStream_t st) {
  widen_kernel<<<elt_blocks(total), kEltThreads, 0, st>>>(a, b, total);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_norms(CgState* S, const double* r64, const float* B, float* rf,
                                int64_t n_pad, int w_pad, int w, double* red, cudaStream_t st) {
  refine_norms_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, r64, B, rf, n_pad, w_pad, w, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_update(double* x64, const float* X, int64_t n_pad, int w_pad, int w,
                                 cudaStream_t st) {
  refine_update_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(x64, X, n_pad, w_pad, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_out(const double* x64, float* Xsol, int64_t n, int w_pad, int w,
                              cudaStream_t st) {
  refine_out_kernel<<<elt_blocks(n * w), kEltThreads, 0, st>>>(x64, Xsol, n, w_pad, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cross_cols(const float* X, int64_t n, int d, const float* Xs, int w, int kernel,
                              const double* inv_l, double f2, float* B, int64_t n_pad, int w_pad,
                              cudaStream_t st) {
  DimScales sc{};
  for (int t = 0; t < d && t < GP_MAX_DIM; ++t) sc.v[t] = static_cast<float>(inv_l[t]);
  cross_cols_kernel<<<elt_blocks(n_pad * w_pad), kEltThreads, 0, st>>>(
      X, n, d, Xs, w, kernel, sc, static_cast<float>(f2), B, n_pad, w_pad);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_coldots(CgState* S, const float* A, const float* B, int64_t n_pad, int w_pad,
                           int w, double* red, cudaStream_t st) {
  coldots_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, A, B, n_pad, w_pad, w, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pred_var(CgState* S, const float* B, const float* U, int64_t n_pad, int w_pad,
                            int w, double f2, float* var, double* red, cudaStream_t st) {
  pred_var_kernel<<<red_blocks(n_pad), kRedThreads, 0, st>>>(S, B, U, n_pad, w_pad, w, f2, var, red);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_copy_col0(const float* X, float* V, int64_t n_pad, int w_pad, cudaStream_t st) {
  copy_col0_kernel<<<elt_blocks(n_pad), kEltThreads, 0, st>>>(X, V, n_pad, w_pad);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gp
