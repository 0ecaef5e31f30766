// Packed FP32-pair arithmetic: the operations of pair_arith.cuh on two
// independent values at once, each FP32 operation issued as one packed FP32x2
// instruction (add.rn.f32x2 / mul.rn.f32x2 / fma.rn.f32x2 through
// __fadd2_rn, __fmul2_rn, __ffma2_rn).  Every lane performs exactly the
// rounded operations of the scalar function of the same name, so each lane's
// result equals the scalar result bit for bit; only the parts that have no
// packed form (round-to-integer, the integer exponent arithmetic, the table
// lookups, square root and reciprocal) run per lane.  Halving the issued
// instructions matters where the scalar form is bound by instruction issue
// (the compensated residual of iterative refinement).
#pragma once

#include "pair_arith.cuh"

namespace gp {
namespace pa2 {

using f2 = float2;

__device__ __forceinline__ f2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
// a - b, rounded once: fma(b, -1, a).
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return __ffma2_rn(b, bc(-1.0f), a); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma_(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 neg(f2 a) { return make_float2(-a.x, -a.y); }

struct fp2 {
  f2 hi, lo;
};

__device__ __forceinline__ fp2 two_sum(f2 a, f2 b) {
  const f2 s = add(a, b);
  const f2 bp = sub(s, a);
  const f2 ap = sub(s, bp);
  return {s, add(sub(a, ap), sub(b, bp))};
}

__device__ __forceinline__ fp2 fast_two_sum(f2 a, f2 b) {
  const f2 s = add(a, b);
  return {s, sub(b, sub(s, a))};
}

__device__ __forceinline__ fp2 two_prod(f2 a, f2 b) {
  const f2 p = mul(a, b);
  return {p, fma_(a, b, neg(p))};
}

__device__ __forceinline__ fp2 add_f(fp2 x, f2 b) {
  const fp2 s = two_sum(x.hi, b);
  return fast_two_sum(s.hi, add(x.lo, s.lo));
}

__device__ __forceinline__ fp2 add_same_sign(fp2 x, fp2 y) {
  const fp2 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, add(s.lo, add(x.lo, y.lo)));
}

__device__ __forceinline__ fp2 add(fp2 x, fp2 y) {
  const fp2 s = two_sum(x.hi, y.hi);
  const fp2 t = two_sum(x.lo, y.lo);
  const fp2 u = fast_two_sum(s.hi, add(s.lo, t.hi));
  return fast_two_sum(u.hi, add(u.lo, t.lo));
}

__device__ __forceinline__ fp2 neg(fp2 x) { return {neg(x.hi), neg(x.lo)}; }

__device__ __forceinline__ fp2 mul(fp2 x, fp2 y) {
  const fp2 p = two_prod(x.hi, y.hi);
  const f2 t = fma_(x.lo, y.hi, mul(x.hi, y.lo));
  return fast_two_sum(p.hi, add(p.lo, t));
}

// Lane c of the pair value x.
__device__ __forceinline__ pa::fpair lane(const fp2& x, int c) {
  return c == 0 ? pa::fpair{x.hi.x, x.lo.x} : pa::fpair{x.hi.y, x.lo.y};
}

// Zero the lanes whose flag is false.
__device__ __forceinline__ fp2 keep(fp2 v, bool k0, bool k1) {
  return {make_float2(k0 ? v.hi.x : 0.0f, k1 ? v.hi.y : 0.0f),
          make_float2(k0 ? v.lo.x : 0.0f, k1 ? v.lo.y : 0.0f)};
}

// pa::exp on two lanes (see pair_arith.cuh for the method).
__device__ __forceinline__ fp2 exp(fp2 u, const pa::ExpConsts& C) {
  const bool live0 = !(u.hi.x < pa::kExpLow), live1 = !(u.hi.y < pa::kExpLow);
  const f2 m0 = mul(u.hi, bc(C.inv_ln2_64));
  // Lanes that the scalar form returns early for get a harmless k here and are
  // zeroed at the end.
  const f2 kf = make_float2(live0 ? rintf(m0.x) : 0.0f, live1 ? rintf(m0.y) : 0.0f);
  const int k0 = static_cast<int>(kf.x), k1 = static_cast<int>(kf.y);
  const fp2 r0 = two_sum(u.hi, neg(mul(kf, bc(C.c0))));
  const fp2 p1 = two_prod(kf, bc(C.c1));
  const fp2 r1 = two_sum(r0.hi, neg(p1.hi));
  const f2 small = sub(sub(add(r0.lo, r1.lo), p1.lo), mul(kf, bc(C.c2)));
  const fp2 r2 = two_sum(r1.hi, u.lo);
  const fp2 r = two_sum(r2.hi, add(r2.lo, small));
  const f2 h = r.hi, rl = r.lo;
  f2 t = fma_(h, bc(1.0f / 120.0f), bc(1.0f / 24.0f));
  t = fma_(h, t, bc(1.0f / 6.0f));
  const f2 h2 = mul(h, h);
  const f2 q = mul(mul(h2, h), t);
  const fp2 sq = two_prod(h, h);
  const f2 s2l = fma_(rl, fma_(bc(0.5f), h2, h), mul(bc(0.5f), sq.lo));
  const fp2 a = fast_two_sum(bc(1.0f), h);
  const fp2 b = fast_two_sum(a.hi, mul(bc(0.5f), sq.hi));
  const f2 lo = add(add(add(q, add(rl, s2l)), a.lo), b.lo);
  const fp2 er = fast_two_sum(b.hi, lo);
  const int j0 = k0 & 63, j1 = k1 & 63;
  const fp2 tab{make_float2(C.hi[j0], C.hi[j1]), make_float2(C.lo[j0], C.lo[j1])};
  const fp2 v = mul(er, tab);
  const f2 sc = make_float2(pa::bits_to_float(static_cast<uint32_t>((k0 >> 6) + 127) << 23),
                            pa::bits_to_float(static_cast<uint32_t>((k1 >> 6) + 127) << 23));
  return keep({mul(v.hi, sc), mul(v.lo, sc)}, live0, live1);
}

// pa::sqrt on two lanes.
__device__ __forceinline__ fp2 sqrt(fp2 x) {
  const bool pos0 = x.hi.x > 0.0f, pos1 = x.hi.y > 0.0f;
  const f2 s = make_float2(pos0 ? __fsqrt_rn(x.hi.x) : 1.0f, pos1 ? __fsqrt_rn(x.hi.y) : 1.0f);
  const fp2 p = two_prod(s, s);
  const f2 res = add(sub(sub(x.hi, p.hi), p.lo), x.lo);
  const f2 rc = make_float2(__frcp_rn(s.x), __frcp_rn(s.y));
  return keep(fast_two_sum(s, mul(res, mul(bc(0.5f), rc))), pos0, pos1);
}

// pa::sqdist of the row point xi against the column points xa (lane 0) and xb (lane 1).
template <int DMAX>
__device__ __forceinline__ fp2 sqdist(const float* xi, const float* xa, const float* xb, int d) {
  fp2 acc{bc(0.0f), bc(0.0f)};
  for (int t = 0; t < DMAX && t < d; ++t) {
    const fp2 df = two_sum(bc(xi[t]), make_float2(-xa[t], -xb[t]));
    const fp2 p = two_prod(df.hi, df.hi);
    const fp2 sq = fast_two_sum(p.hi, fma_(add(df.hi, df.hi), df.lo, p.lo));
    acc = t == 0 ? sq : add_same_sign(acc, sq);
  }
  return acc;
}

// pa::kernel_entry on two lanes.
__device__ __forceinline__ fp2 kernel_entry(fp2 r2, int kernel, pa::fpair kc, const pa::ExpConsts& C) {
  const fp2 k2{bc(kc.hi), bc(kc.lo)};
  if (kernel == 0) return exp(neg(mul(r2, k2)), C);
  const fp2 a = mul(sqrt(r2), k2);
  return mul(add_f(a, bc(1.0f)), exp(neg(a), C));
}

}  // namespace pa2
}  // namespace gp
