// Double-float ("FP32 pair") arithmetic for the compensated residual of
// mixed-precision iterative refinement.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits, built from error-free transformations of IEEE
// FP32 operations:
//  - TwoSum (Knuth, The Art of Computer Programming vol. 2, §4.2.2): s + e = a + b
//    exactly, for any a, b.  FastTwoSum (Dekker 1971): the same in three
//    operations when |a| >= |b|.
//  - TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p), so that
//    p + e = a b exactly.
//  - Pair sums and products: the double-word algorithms analysed by Joldes,
//    Muller and Popescu ("Tight and rigorous error bounds for basic building
//    blocks of double-word arithmetic", ACM TOMS 44(2), 2017): DWPlusFP,
//    SloppyDWPlusDW (used only for operands of one sign), AccurateDWPlusDW,
//    DWTimesFP and DWTimesDW.
//  - exp: Tang's table-driven method (ACM TOMS 15(2), 1989).  u = (64 m + j)
//    ln2/64 + r with |r| <= ln2/128 + tiny, exp(u) = 2^m 2^(j/64) e^r; the
//    reduction subtracts k ln2/64 in Cody & Waite's manner, with ln2/64 split
//    into three floats c0 + c1 + c2 (c0 of 11 significant bits, so that k c0
//    is exact for |k| < 2^13), and e^r is its Taylor series to degree 5
//    (the first omitted term is below 4e-17).  The 64 table values 2^(j/64)
//    are formed on the host in FP64 and split into pairs.
//  - sqrt: the correctly rounded FP32 square root with one Newton correction
//    in pair arithmetic (Karp and Markstein, ACM TOMS 23(4), 1997).
// Every operation is an explicitly rounded IEEE operation, so a host build
// (no FP contraction) gives the same bits as the device.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace gp {

#ifdef __CUDACC__
#define GP_PHD __host__ __device__ __forceinline__
#else
#define GP_PHD inline
#endif

namespace pa {

struct fpair {
  float hi, lo;
};

GP_PHD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
GP_PHD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
GP_PHD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
GP_PHD float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
GP_PHD float sqrt_(float a) {
#ifdef __CUDA_ARCH__
  return __fsqrt_rn(a);
#else
  return sqrtf(a);
#endif
}
GP_PHD float rcp_(float a) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(a);
#else
  return 1.0f / a;
#endif
}
// Round to the nearest integer, ties to even (the default rounding mode).
GP_PHD float rint_(float a) {
#ifdef __CUDA_ARCH__
  return rintf(a);
#else
  return nearbyintf(a);
#endif
}
GP_PHD float bits_to_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
#endif
}

GP_PHD fpair two_sum(float a, float b) {
  const float s = add(a, b);
  const float bp = sub(s, a);
  const float ap = sub(s, bp);
  return {s, add(sub(a, ap), sub(b, bp))};
}

// Requires |a| >= |b| (or a == 0).
GP_PHD fpair fast_two_sum(float a, float b) {
  const float s = add(a, b);
  return {s, sub(b, sub(s, a))};
}

GP_PHD fpair two_prod(float a, float b) {
  const float p = mul(a, b);
  return {p, fma_(a, b, -p)};
}

// DWPlusFP: x + b.
GP_PHD fpair add_f(fpair x, float b) {
  const fpair s = two_sum(x.hi, b);
  return fast_two_sum(s.hi, add(x.lo, s.lo));
}

// SloppyDWPlusDW: x + y for x, y of the same sign.
GP_PHD fpair add_same_sign(fpair x, fpair y) {
  const fpair s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, add(s.lo, add(x.lo, y.lo)));
}

// AccurateDWPlusDW: x + y for any signs.
GP_PHD fpair add(fpair x, fpair y) {
  const fpair s = two_sum(x.hi, y.hi);
  const fpair t = two_sum(x.lo, y.lo);
  fpair u = fast_two_sum(s.hi, add(s.lo, t.hi));
  return fast_two_sum(u.hi, add(u.lo, t.lo));
}

GP_PHD fpair neg(fpair x) { return {-x.hi, -x.lo}; }

// DWTimesFP: x b.
GP_PHD fpair mul_f(fpair x, float b) {
  const fpair p = two_prod(x.hi, b);
  return fast_two_sum(p.hi, fma_(x.lo, b, p.lo));
}

// DWTimesDW: x y.
GP_PHD fpair mul(fpair x, fpair y) {
  const fpair p = two_prod(x.hi, y.hi);
  const float t = fma_(x.lo, y.hi, mul(x.hi, y.lo));
  return fast_two_sum(p.hi, add(p.lo, t));
}

// Nearest pair of an FP64 value (exact when the value has <= 48 significant bits).
GP_PHD fpair from_double(double v) {
  const float hi = static_cast<float>(v);
  return {hi, static_cast<float>(v - static_cast<double>(hi))};
}
GP_PHD double to_double(fpair x) { return static_cast<double>(x.hi) + static_cast<double>(x.lo); }

// Constants of the pair exponential and the kernel evaluation (host-built).
struct ExpConsts {
  float hi[64], lo[64];   // 2^(j/64) = hi[j] + lo[j]
  float inv_ln2_64;       // 64 / ln2 (rounded; only picks k)
  float c0, c1, c2;       // ln2 / 64 = c0 + c1 + c2, c0 with 11 significant bits
};

// Arguments below this give a result under 2^-125 (treated as 0: absolute error < 3e-38).
constexpr float kExpLow = -86.0f;

// exp(u) for u <= 0 (|u| <= 88 for positive u is also exact to the same error).
GP_PHD fpair exp(fpair u, const ExpConsts& C) {
  if (u.hi < kExpLow) return {0.0f, 0.0f};
  const float kf = rint_(mul(u.hi, C.inv_ln2_64));   // |k| <= 7941
  const int k = static_cast<int>(kf);
  // r = u - k (c0 + c1 + c2): k c0 is exact; each subtraction is error-free.
  const fpair r0 = two_sum(u.hi, -mul(kf, C.c0));
  const fpair p1 = two_prod(kf, C.c1);
  const fpair r1 = two_sum(r0.hi, -p1.hi);
  const float small = sub(sub(add(r0.lo, r1.lo), p1.lo), mul(kf, C.c2));
  const fpair r2 = two_sum(r1.hi, u.lo);
  const fpair r = two_sum(r2.hi, add(r2.lo, small));
  // e^r = 1 + r + r^2/2 + r^3/6 + r^4/24 + r^5/120.
  const float h = r.hi, rl = r.lo;
  float t = fma_(h, 1.0f / 120.0f, 1.0f / 24.0f);
  t = fma_(h, t, 1.0f / 6.0f);
  const float h2 = mul(h, h);
  const float q = mul(mul(h2, h), t);                  // r^3/6 + r^4/24 + r^5/120
  const fpair sq = two_prod(h, h);                     // r^2 = sq.hi + sq.lo (of h)
  const float s2l = fma_(rl, fma_(0.5f, h2, h), mul(0.5f, sq.lo));   // lo parts of r^2/2, r^3/6
  const fpair a = fast_two_sum(1.0f, h);
  const fpair b = fast_two_sum(a.hi, mul(0.5f, sq.hi));
  const float lo = add(add(add(q, add(rl, s2l)), a.lo), b.lo);
  const fpair er = fast_two_sum(b.hi, lo);
  // 2^(j/64) e^r, then the exact scaling by 2^m.
  const int j = k & 63;
  const int m = k >> 6;                                // floor(k / 64)
  const fpair v = mul(er, fpair{C.hi[j], C.lo[j]});
  const float sc = bits_to_float(static_cast<uint32_t>(m + 127) << 23);
  return {mul(v.hi, sc), mul(v.lo, sc)};
}

// sqrt(x) for x >= 0.
GP_PHD fpair sqrt(fpair x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float s = sqrt_(x.hi);
  const fpair p = two_prod(s, s);
  // x - s^2 exactly up to the rounding of the sum of small terms, over 2 s.
  const float res = add(sub(sub(x.hi, p.hi), p.lo), x.lo);
  return fast_two_sum(s, mul(res, mul(0.5f, rcp_(s))));
}

// Squared distance between two FP32 points, in pair arithmetic (the
// differences are exact pairs; the sum has only non-negative terms).
template <int DMAX>
GP_PHD fpair sqdist(const float* xi, const float* xj, int d) {
  fpair acc{0.0f, 0.0f};
  for (int t = 0; t < DMAX && t < d; ++t) {
    const fpair df = two_sum(xi[t], -xj[t]);
    const fpair p = two_prod(df.hi, df.hi);
    const fpair sq = fast_two_sum(p.hi, fma_(add(df.hi, df.hi), df.lo, p.lo));
    acc = t == 0 ? sq : add_same_sign(acc, sq);
  }
  return acc;
}

// Kernel entry k(r) from r^2: Gaussian exp(-r^2 kc) with kc = 1/(2 l^2);
// Matern-3/2 (1 + a) exp(-a) with a = r kc, kc = sqrt(3)/l.
GP_PHD fpair kernel_entry(fpair r2, int kernel, fpair kc, const ExpConsts& C) {
  if (kernel == 0) return exp(neg(mul(r2, kc)), C);
  const fpair a = mul(sqrt(r2), kc);
  return mul(add_f(a, 1.0f), exp(neg(a), C));
}

// Host: fill the exponential constants: the table from the FP64 library exp2,
// split into pairs; ln2/64 from the long-double logarithm (at least 64
// significant bits), split into three floats.
inline void make_exp_consts(ExpConsts& C) {
  for (int j = 0; j < 64; ++j) {
    const double v = exp2(static_cast<double>(j) / 64.0);
    const fpair p = from_double(v);
    C.hi[j] = p.hi;
    C.lo[j] = p.lo;
  }
  const long double ln2_64 = logl(2.0L) / 64.0L;
  C.inv_ln2_64 = static_cast<float>(1.0L / ln2_64);
  // c0: ln2/64 rounded to 11 significant bits (clear the low 13 of 24).
  float c0f = static_cast<float>(ln2_64);
  uint32_t u;
  memcpy(&u, &c0f, sizeof u);
  u &= ~0x1FFFu;
  memcpy(&c0f, &u, sizeof u);
  C.c0 = c0f;
  const long double rem = ln2_64 - static_cast<long double>(c0f);
  C.c1 = static_cast<float>(rem);
  C.c2 = static_cast<float>(rem - static_cast<long double>(C.c1));
}

// Host: the kernel constant kc as a pair.
inline fpair kernel_pair_const(int kernel, double l) {
  return from_double(kernel == 0 ? 1.0 / (2.0 * l * l) : ::sqrt(3.0) / l);
}

}  // namespace pa
}  // namespace gp
