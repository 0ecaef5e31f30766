"""Host build of the device's FP32-pair arithmetic (csrc/pair_arith.cuh).

The compensated residual of iterative refinement evaluates kernel entries in
double-float arithmetic on the FP32 pipe.  Every operation there is an
explicitly rounded IEEE FP32 operation, so the header compiled for the host
(g++, no FP contraction) performs the same arithmetic as the device.  These
tests pin it against high-precision values (mpmath, 40 digits) from the
definitions: exp, sqrt, the squared distance of two FP32 points and the
Gaussian / Matern-3/2 entries over the argument ranges of the workloads.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2503_02259_gb300", "csrc", "pair_arith.cuh")

mp = pytest.importorskip("mpmath")
mp.mp.dps = 40

SRC = r'''
#include "%s"
using namespace gp::pa;
static ExpConsts C;
extern "C" void init() { make_exp_consts(C); }
extern "C" void pexp(const double* u, double* out, int n) {
  for (int i = 0; i < n; ++i) out[i] = to_double(gp::pa::exp(from_double(u[i]), C));
}
extern "C" void psqrt(const double* x, double* out, int n) {
  for (int i = 0; i < n; ++i) out[i] = to_double(gp::pa::sqrt(from_double(x[i])));
}
extern "C" void psqdist(const float* a, const float* b, int d, int n, double* out) {
  for (int i = 0; i < n; ++i) out[i] = to_double(sqdist<16>(a + i * d, b + i * d, d));
}
extern "C" void pentry(const float* a, const float* b, int d, int n, int kernel, double l,
                       double* out) {
  const fpair kc = kernel_pair_const(kernel, l);
  for (int i = 0; i < n; ++i)
    out[i] = to_double(kernel_entry(sqdist<16>(a + i * d, b + i * d, d), kernel, kc, C));
}
extern "C" void consts(float* c) { c[0] = C.c0; c[1] = C.c1; c[2] = C.c2; c[3] = C.inv_ln2_64; }
'''


@pytest.fixture(scope="module")
def P(tmp_path_factory):
    d = tmp_path_factory.mktemp("pair")
    src = d / "pair.cpp"
    src.write_text(SRC % HDR)
    so = d / "pair.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", str(src),
                    "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.init()
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _run(L, name, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    getattr(L, name)(_p(x), _p(out), x.size)
    return out


def _pair_value(v):
    """The pair the device forms from an FP64 value (hi = fl32(v), lo = fl32(v - hi))."""
    hi = np.float32(v)
    lo = np.float32(v - np.float64(hi))
    return mp.mpf(float(hi)) + mp.mpf(float(lo))


def test_split_constants_are_exact_pieces_of_ln2_over_64(P):
    c = np.empty(4, dtype=np.float32)
    P.consts(_p(c))
    c0, c1, c2 = (mp.mpf(float(v)) for v in c[:3])
    # c0 has at most 11 significant bits, so k c0 is exact for |k| < 2^13.
    m, e = np.frexp(np.float64(c[0]))
    assert float(m * 2 ** 11) == int(m * 2 ** 11)
    err = abs(c0 + c1 + c2 - mp.log(2) / 64) / (mp.log(2) / 64)
    assert err < 1e-17


def test_exp_over_the_reduced_argument_range(P):
    rng = np.random.default_rng(0)
    u = np.concatenate([-rng.uniform(0, 86, 4000), -rng.uniform(0, 1, 1000),
                        -rng.uniform(0, 1e-3, 200), [0.0, -1e-30, -86.0]])
    # Arguments at and next to the reduction's breakpoints k ln2 / 128.
    k = np.arange(0, 11000, 37)
    br = -k * np.log(2) / 128
    u = np.concatenate([u, br, np.nextafter(br, 0), np.nextafter(br, -1)])
    u = u[u >= -86.0]
    got = _run(P, "pexp", u)
    worst = worst_abs = 0.0
    for ui, g in zip(u, got):
        ref = mp.exp(_pair_value(ui))
        if ref > mp.mpf(2) ** -100:
            worst = max(worst, float(abs(mp.mpf(g) - ref) / ref))
        else:
            # The low word is subnormal below ~2^-102: absolute accuracy only.
            worst_abs = max(worst_abs, float(abs(mp.mpf(g) - ref)))
    assert worst < 2e-14, worst   # about 6 u^2, u = 2^-24 (median 1.2e-15)
    assert worst_abs < 2.0 ** -140, worst_abs


def test_exp_below_the_cutoff_is_zero(P):
    got = _run(P, "pexp", np.array([-86.5, -100.0, -1e4]))
    assert np.all(got == 0.0)


def test_exp_rejects_a_plausible_mistake(P):
    # Dropping the pair's low word of the argument costs about |u| 2^-24 of
    # relative accuracy: the implementation must be far better than that.
    u = -np.linspace(1.0, 69.0, 200) - 1e-9
    got = _run(P, "pexp", u)
    for ui, g in zip(u, got):
        ref = mp.exp(_pair_value(ui))
        hi_only = mp.exp(mp.mpf(float(np.float32(ui))))   # the argument's high word alone
        e_got = abs(mp.mpf(g) - ref) / ref
        e_hi = abs(hi_only - ref) / ref
        assert e_got < 2e-14 and (e_hi == 0 or e_got < 1e-3 * e_hi)


def test_sqrt(P):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(0, 1, 2000), 10 ** rng.uniform(-12, 3, 2000), [0.0, 1.0, 4.0]])
    got = _run(P, "psqrt", x)
    for xi, g in zip(x, got):
        ref = mp.sqrt(_pair_value(xi))
        if ref == 0:
            assert g == 0.0
        else:
            assert abs(mp.mpf(g) - ref) / ref < 2e-14


@pytest.mark.parametrize("d", [1, 2, 3, 8, 16])
def test_squared_distance_of_fp32_points(P, d):
    rng = np.random.default_rng(d)
    n = 500
    a = rng.uniform(-1, 1, (n, d)).astype(np.float32)
    b = (a + rng.normal(0, 10.0 ** rng.uniform(-6, 0, (n, 1)), (n, d))).astype(np.float32)
    out = np.empty(n)
    P.psqdist(_p(a), _p(b), d, n, _p(out))
    for i in range(n):
        ref = mp.fsum((mp.mpf(float(a[i, t])) - mp.mpf(float(b[i, t]))) ** 2 for t in range(d))
        if ref == 0:
            assert out[i] == 0.0
        else:
            assert abs(mp.mpf(out[i]) - ref) / ref < 1e-14


# (kernel, l, d, coordinate spread) of the workloads: the small problem, the
# fused matvec problem, the precision problem and the differentiation problem.
CASES = [(0, 0.3, 3, 1.0), (1, 0.2, 3, 1.0), (0, 0.05, 2, 1.0), (0, 1.2, 8, 0.5), (1, 0.05, 2, 0.2)]


@pytest.mark.parametrize("kernel,l,d,spread", CASES)
def test_kernel_entries_match_the_definition(P, kernel, l, d, spread):
    rng = np.random.default_rng(int(100 * l) + d)
    n = 600
    a = (spread * rng.uniform(0, 1, (n, d))).astype(np.float32)
    b = (a + l * rng.normal(0, 10.0 ** rng.uniform(-3, 0.7, (n, 1)), (n, d))).astype(np.float32)
    b[:5] = a[:5]                                       # r = 0: k = 1
    out = np.empty(n)
    P.pentry(_p(a), _p(b), d, n, kernel, ctypes.c_double(l), _p(out))
    L = mp.mpf(l)
    for i in range(n):
        r2 = mp.fsum((mp.mpf(float(a[i, t])) - mp.mpf(float(b[i, t]))) ** 2 for t in range(d))
        if kernel == 0:
            ref = mp.exp(-r2 / (2 * L * L))
        else:
            aa = mp.sqrt(3 * r2) / L
            ref = (1 + aa) * mp.exp(-aa)
        if ref > 1e-29:
            # The argument u (r^2 / (2 l^2) or sqrt(3) r / l) carries a few
            # 2^-48 of relative error from the pair sum, the pair constant and
            # the pair product; exp turns it into |u| times that.
            tol = 2e-14 + 4e-14 * float(abs(mp.log(ref)))
            assert abs(mp.mpf(out[i]) - ref) / ref < tol, (i, out[i], ref)
        else:
            assert abs(out[i] - float(ref)) < 1e-37
    assert np.all(out[:5] == 1.0)
