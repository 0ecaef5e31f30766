"""Pins for the FP64 oracle against facts fixed outside the oracle itself:
published test vectors, closed forms, finite differences, brute force,
spectral (Bochner) representations and statistical bands.

CPU only; the whole file runs in well under a minute.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2503_02259_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- probes --

def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for row in rows:
        state = int(row[0])
        for expect in row[1:]:
            state, out = O.splitmix64_next(state)
            assert out == int(expect)


def test_rademacher_matches_scalar_definition():
    n, p, seed = 37, 5, 0xC0FFEE
    Z = O.rademacher_probes(n, p, seed)
    for c in range(p):
        for i in range(n):
            h = O.probe_hash(seed, c, i)
            assert Z[i, c] == (1.0 if (h >> 63) == 0 else -1.0)


def test_rademacher_balance():
    Z = O.rademacher_probes(20000, 4, 3)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    # Each column is a fair coin: mean within 4 sigma of 0.
    assert np.all(np.abs(Z.mean(axis=0)) < 4.0 / math.sqrt(20000))
    # Columns differ from one another (the column index enters the hash).
    assert np.abs(Z[:, 0] @ Z[:, 1]) < 4.0 * math.sqrt(20000)


# ---------------------------------------------------------------- kernels --

def _bochner_gaussian(delta, l, nsamp, rng):
    # k(r) = E[cos(w . delta)], w ~ N(0, I / l^2)  (spectral density of the RBF kernel)
    w = rng.standard_normal((nsamp, delta.size)) / l
    return float(np.mean(np.cos(w @ delta)))


def _bochner_matern32(delta, l, nsamp, rng):
    # Matern-nu spectral density ~ (2 nu / l^2 + |w|^2)^-(nu + d/2): a multivariate
    # Student-t with 2 nu = 3 degrees of freedom and scale 1 / l.
    g = rng.standard_normal((nsamp, delta.size))
    u = rng.chisquare(3.0, size=(nsamp, 1))
    w = g / (l * np.sqrt(u / 3.0))
    return float(np.mean(np.cos(w @ delta)))


@pytest.mark.parametrize("kind,sampler", [(O.GAUSSIAN, _bochner_gaussian),
                                          (O.MATERN32, _bochner_matern32)])
def test_kernel_matches_spectral_representation(kind, sampler):
    rng = np.random.default_rng(11)
    l = 0.7
    for d in (1, 3):
        for r in (0.0, 0.3, 0.7, 1.5):
            delta = np.zeros(d)
            delta[0] = r
            mc = sampler(delta, l, 400_000, rng)
            k = O.kernel_value(np.array(r * r), kind, l)
            assert abs(mc - k) < 6e-3, (kind, d, r, mc, k)


def test_gaussian_is_separable_over_dimensions():
    rng = np.random.default_rng(1)
    A = rng.random((7, 4))
    B = rng.random((5, 4))
    l = 0.4
    full = O.kernel_value(O.sqdist(A, B), O.GAUSSIAN, l)
    prod = np.ones_like(full)
    for t in range(4):
        prod *= O.kernel_value(O.sqdist(A[:, t:t + 1], B[:, t:t + 1]), O.GAUSSIAN, l)
    np.testing.assert_allclose(full, prod, rtol=1e-13)


def test_sqdist_brute_force():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((6, 3))
    B = rng.standard_normal((4, 3))
    R2 = O.sqdist(A, B)
    for i in range(6):
        for j in range(4):
            assert R2[i, j] == pytest.approx(sum((A[i, t] - B[j, t]) ** 2 for t in range(3)), rel=1e-14)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_kernel_dl_central_difference(kind):
    r2 = np.array([1e-4, 0.01, 0.09, 0.3, 1.0, 2.5])
    for l in (0.2, 0.7, 1.3):
        h = 1e-5 * l
        fd = (O.kernel_value(r2, kind, l + h) - O.kernel_value(r2, kind, l - h)) / (2 * h)
        np.testing.assert_allclose(O.kernel_dl(r2, kind, l), fd, rtol=1e-7, atol=1e-13)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_kernel_special_cases(kind):
    assert O.kernel_value(np.array(0.0), kind, 0.3) == 1.0
    assert O.kernel_dl(np.array(0.0), kind, 0.3) == 0.0
    far = np.array((40 * 0.3) ** 2)
    assert O.kernel_value(far, kind, 0.3) < 1e-25
    assert O.kernel_dl(far, kind, 0.3) < 1e-20


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_khat_symmetric_positive_definite(kind):
    X = inputs.points(300, 3, seed=5)
    theta = (0.05, 1.3, 0.25)
    Kh = O.khat_dense(X, kind, theta)
    assert np.array_equal(Kh, Kh.T)
    assert np.linalg.eigvalsh(Kh).min() >= theta[0] * (1 - 1e-10)


# -------------------------------------------------------------- the matvec --

def _identical_points(n, d, value=0.37):
    return np.full((n, d), value, dtype=np.float32)


def _far_points(n, d, spacing):
    X = np.zeros((n, d), dtype=np.float32)
    X[:, 0] = spacing * np.arange(n)
    return X


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_kmv_identical_points_closed_form(kind):
    n, s, f, l = 50, 0.2, 1.7, 0.3
    V = inputs.gaussian_block(n, 3, seed=1).astype(np.float64)
    Y, dYf, dYl = O.kmv_rows(_identical_points(n, 2), V, kind, (s, f, l), block=16)
    colsum = V.sum(axis=0)
    np.testing.assert_allclose(Y, f * f * colsum[None, :] + s * V, rtol=1e-13)
    np.testing.assert_allclose(dYf, 2 * f * np.repeat(colsum[None, :], n, 0), rtol=1e-13)
    np.testing.assert_allclose(dYl, 0.0, atol=1e-15)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_kmv_far_points_closed_form(kind):
    n, s, f, l = 40, 0.2, 1.7, 0.1
    V = inputs.gaussian_block(n, 2, seed=2).astype(np.float64)
    Y, dYf, dYl = O.kmv_rows(_far_points(n, 3, 40 * l), V, kind, (s, f, l))
    np.testing.assert_allclose(Y, (f * f + s) * V, rtol=1e-12)
    np.testing.assert_allclose(dYf, 2 * f * V, rtol=1e-12)
    np.testing.assert_allclose(dYl, 0.0, atol=1e-12)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_kmv_rows_brute_force(kind):
    n, theta = 60, (0.1, 1.2, 0.35)
    X = inputs.points(n, 3, seed=9)
    V = inputs.gaussian_block(n, 4, seed=3).astype(np.float64)
    rows = np.array([0, 7, 59, 13])
    Y, dYf, dYl = O.kmv_rows(X, V, kind, theta, rows=rows, block=3)
    s, f, l = theta
    Xd = X.astype(np.float64)
    for a, i in enumerate(rows):
        for c in range(4):
            acc_k = acc_d = 0.0
            for j in range(n):
                r2 = float(np.sum((Xd[i] - Xd[j]) ** 2))
                acc_k += float(O.kernel_value(np.array(r2), kind, l)) * V[j, c]
                acc_d += float(O.kernel_dl(np.array(r2), kind, l)) * V[j, c]
            assert Y[a, c] == pytest.approx(f * f * acc_k + s * V[i, c], rel=1e-12, abs=1e-13)
            assert dYf[a, c] == pytest.approx(2 * f * acc_k, rel=1e-12, abs=1e-13)
            assert dYl[a, c] == pytest.approx(f * f * acc_d, rel=1e-12, abs=1e-13)


def test_predict_mean_identical_points_closed_form():
    n, s, f, l = 30, 0.3, 1.1, 0.5
    X = _identical_points(n, 3)
    y = inputs.gaussian_block(n, 1, seed=4)[:, 0].astype(np.float64)
    alpha = O.exact_nll(X, y, O.GAUSSIAN, (s, f, l))["alpha"]
    mu = O.predict_mean(X, X[:2], alpha, O.GAUSSIAN, (s, f, l))
    np.testing.assert_allclose(mu, f * f * y.sum() / (s + n * f * f), rtol=1e-12)


def test_predict_mean_interpolates_at_small_noise():
    X = inputs.points(40, 2, seed=12)
    y = np.sin(3 * X[:, 0].astype(np.float64))
    theta = (1e-8, 1.0, 0.3)
    alpha = O.exact_nll(X, y, O.GAUSSIAN, theta)["alpha"]
    mu = O.predict_mean(X, X, alpha, O.GAUSSIAN, theta)
    np.testing.assert_allclose(mu, y, atol=1e-5)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_predict_var_identical_points_closed_form(kind):
    # All n training points at x0: Kh = f^2 1 1^T + s I.  A test point at distance r
    # has k_c = f^2 k(r) 1, and Sherman-Morrison gives
    # var = f^2 - f^4 k(r)^2 n / (s + n f^2).
    n, s, f, l = 30, 0.3, 1.1, 0.5
    X = _identical_points(n, 3)
    r = np.array([0.0, 0.2, 0.7, 1.9])
    Xs = np.repeat(X[:1].astype(np.float64), r.size, axis=0)
    Xs[:, 0] += r
    var = O.predict_var(X, Xs, kind, (s, f, l))
    kr = O.kernel_value(r * r, kind, l)
    np.testing.assert_allclose(var, f * f - f ** 4 * kr * kr * n / (s + n * f * f), rtol=1e-10)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_predict_var_far_points_is_the_prior(kind):
    # Test points far from every training point (>= 40 l): k_c = 0, var = f^2.
    X = inputs.points(50, 2, seed=31)
    Xs = inputs.points(6, 2, seed=32).astype(np.float64) + 40.0
    theta = (0.2, 1.3, 0.4)
    np.testing.assert_allclose(O.predict_var(X, Xs, kind, theta), theta[1] ** 2, rtol=1e-12)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_predict_var_is_the_joint_gaussian_conditional(kind):
    # Brute force from the joint covariance C of (y, y*) (Cov(y) = Kh,
    # Cov(y, y*) = f^2 K(X, X*), Cov(y*) = f^2 K(X*, X*)): the conditional
    # covariance of y* given y is the inverse of the (y*, y*) block of C^-1.
    X = inputs.points(25, 2, seed=33)
    Xs = inputs.points(7, 2, seed=34)
    theta = (0.15, 0.9, 0.3)
    s, f, l = theta
    Kc = f * f * O.kernel_value(O.sqdist(X, Xs), kind, l)
    C = np.block([[O.khat_dense(X, kind, theta), Kc],
                  [Kc.T, f * f * O.kernel_value(O.sqdist(Xs, Xs), kind, l)]])
    post = np.linalg.inv(np.linalg.inv(C)[25:, 25:])
    var = O.predict_var(X, Xs, kind, theta)
    np.testing.assert_allclose(var, np.diag(post), rtol=1e-7)
    assert np.all(var > 0) and np.all(var <= f * f)


# --------------------------------------------------------- exact NLL / grad --

@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_exact_nll_identical_points_closed_form(kind):
    n, s, f, l = 25, 0.15, 0.9, 0.4
    X = _identical_points(n, 3)
    y = inputs.gaussian_block(n, 1, seed=6)[:, 0].astype(np.float64)
    out = O.exact_nll(X, y, kind, (s, f, l))
    lam = s + n * f * f
    alpha = (y - f * f * y.sum() / lam) / s           # Sherman-Morrison
    logdet = math.log(lam) + (n - 1) * math.log(s)
    loss = 0.5 * (y @ alpha + logdet + n * math.log(2 * math.pi))
    g_s = 0.5 * (-(alpha @ alpha) + 1.0 / lam + (n - 1) / s)
    g_f = 0.5 * (-2 * f * alpha.sum() ** 2 + 2 * f * n / lam)
    np.testing.assert_allclose(out["alpha"], alpha, rtol=1e-10)
    assert out["logdet"] == pytest.approx(logdet, rel=1e-12)
    assert out["loss"] == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(out["grad"], [g_s, g_f, 0.0], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_exact_nll_far_points_closed_form(kind):
    n, s, f, l = 30, 0.2, 1.4, 0.1
    X = _far_points(n, 2, 40 * l)
    y = inputs.gaussian_block(n, 1, seed=7)[:, 0].astype(np.float64)
    out = O.exact_nll(X, y, kind, (s, f, l))
    c = f * f + s
    yy = y @ y
    assert out["logdet"] == pytest.approx(n * math.log(c), rel=1e-12)
    assert out["loss"] == pytest.approx(0.5 * (yy / c + n * math.log(c) + n * math.log(2 * math.pi)), rel=1e-12)
    np.testing.assert_allclose(out["grad"], [0.5 * (-yy / c ** 2 + n / c),
                                             0.5 * (-2 * f * yy / c ** 2 + 2 * f * n / c), 0.0],
                               rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_exact_grad_central_difference(kind):
    prob = inputs.uniform_problem(120, 3, kind, (0.1, 1.2, 0.3), seed=4)
    theta = np.array(prob.theta)
    g = O.exact_nll(prob.X, prob.y, kind, theta)["grad"]
    for t in range(3):
        h = 1e-4 * theta[t]
        tp, tm = theta.copy(), theta.copy()
        tp[t] += h
        tm[t] -= h
        fd = (O.exact_nll(prob.X, prob.y, kind, tp)["loss"]
              - O.exact_nll(prob.X, prob.y, kind, tm)["loss"]) / (2 * h)
        assert g[t] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(g).max()), (t, g[t], fd)


def test_exact_logdet_against_eigenvalues():
    X = inputs.points(80, 2, seed=8)
    theta = (0.05, 1.0, 0.2)
    out = O.exact_nll(X, np.ones(80), O.MATERN32, theta)
    ev = np.linalg.eigvalsh(O.khat_dense(X, O.MATERN32, theta))
    assert out["logdet"] == pytest.approx(np.sum(np.log(ev)), rel=1e-11)


# ------------------------------------------------------------------- SLQ --

def test_lanczos_two_distinct_eigenvalues_exact():
    # Identical points: Kh = f^2 11^T + s I has eigenvalues s + n f^2 and s, so a
    # 2-step Gauss rule integrates log exactly: z^T log(Kh) z in closed form.
    n, s, f = 40, 0.3, 0.8
    A = f * f * np.ones((n, n)) + s * np.eye(n)
    z = O.rademacher_probes(n, 1, 17)[:, 0]
    a, b = O.lanczos(A, z, 2)
    est = O.gauss_quadrature_log(a, b, z @ z)
    m = z.sum() ** 2 / n
    exact = math.log(s + n * f * f) * m + math.log(s) * (z @ z - m)
    assert est == pytest.approx(exact, rel=1e-12)


def test_lanczos_full_length_equals_matrix_log():
    X = inputs.points(30, 2, seed=10)
    A = O.khat_dense(X, O.GAUSSIAN, (0.1, 1.0, 0.4))
    z = O.rademacher_probes(30, 1, 2)[:, 0]
    a, b = O.lanczos(A, z, 30)
    ev, U = np.linalg.eigh(A)
    exact = float(z @ (U @ (np.log(ev) * (U.T @ z))))
    assert O.gauss_quadrature_log(a, b, z @ z) == pytest.approx(exact, rel=1e-9)


def test_lanczos_from_cg_matches_explicit_lanczos():
    # The CG step coefficients carry the Lanczos tridiagonal of K from q1 = b/||b||.
    X = inputs.points(200, 3, seed=11)
    A = O.khat_dense(X, O.GAUSSIAN, (0.1, 1.0, 0.3))
    z = O.rademacher_probes(200, 1, 5)[:, 0]
    _, _, _, al, be = O.cg(A, z, 1e-12, 12)
    a1, b1 = O.lanczos_from_cg(al[0], be[0], 10)
    a2, b2 = O.lanczos(A, z, 10)
    np.testing.assert_allclose(a1, a2, rtol=1e-8)
    np.testing.assert_allclose(b1, np.abs(b2), rtol=1e-7)


def test_slq_converges_to_logdet_within_3_sigma():
    X = inputs.points(300, 3, seed=13)
    A = O.khat_dense(X, O.GAUSSIAN, (0.1, 1.0, 0.3))
    exact = np.linalg.slogdet(A)[1]
    Z = O.rademacher_probes(300, 200, 99)
    est, vals = O.slq_logdet(A, Z, 30)
    sigma = vals.std(ddof=1) / math.sqrt(vals.size)
    assert abs(est - exact) < 3 * sigma + 1e-9 * abs(exact)
    # More probes shrink the band at ~1/sqrt(p).
    est_few, vals_few = O.slq_logdet(A, Z[:, :20], 30)
    assert vals_few.std(ddof=1) / math.sqrt(20) > sigma


# ------------------------------------------------------------- Hutchinson --

def test_hutchinson_exact_for_diagonal():
    n, s, f, l = 50, 0.25, 1.3, 0.1
    X = _far_points(n, 2, 40 * l)
    Kh = O.khat_dense(X, O.GAUSSIAN, (s, f, l))
    dKs = O.dkhat_dense(X, O.GAUSSIAN, (s, f, l))
    Z = O.rademacher_probes(n, 3, 4)
    tr, vals = O.hutchinson_traces(Kh, dKs, Z)
    c = f * f + s
    np.testing.assert_allclose(vals[0], n / c, rtol=1e-12)
    np.testing.assert_allclose(vals[1], 2 * f * n / c, rtol=1e-12)
    np.testing.assert_allclose(vals[2], 0.0, atol=1e-12)


def test_hutchinson_unbiased_within_3_sigma():
    prob = inputs.uniform_problem(250, 3, O.MATERN32, (0.1, 1.0, 0.3), seed=14)
    ex = O.exact_nll(prob.X, prob.y, prob.kind, prob.theta)
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    dKs = O.dkhat_dense(prob.X, prob.kind, prob.theta)
    Z = O.rademacher_probes(250, 400, 7)
    tr, vals = O.hutchinson_traces(Kh, dKs, Z)
    sig = vals.std(axis=1, ddof=1) / math.sqrt(400)
    assert np.all(np.abs(tr - ex["trace"]) < 3 * sig + 1e-10)


def test_est_nll_approaches_exact():
    prob = inputs.small_problem(seed=0, n=300)
    ex = O.exact_nll(prob.X, prob.y, prob.kind, prob.theta)
    Z = O.rademacher_probes(300, 256, 1)
    es = O.est_nll(prob.X, prob.y, prob.kind, prob.theta, Z, 30)
    assert es["yalpha"] == pytest.approx(ex["yalpha"], rel=1e-12)
    np.testing.assert_allclose(es["quad"], ex["quad"], rtol=1e-12)
    sig_ld = es["logdet_probes"].std(ddof=1) / 16.0
    assert abs(es["logdet"] - ex["logdet"]) < 3 * sig_ld
    sig_tr = es["trace_probes"].std(axis=1, ddof=1) / 16.0
    assert np.all(np.abs(es["trace"] - ex["trace"]) < 3 * sig_tr + 1e-10)
    # The estimator's loss and gradient differ from the exact ones only through
    # the two estimated terms: L~ - L = (logdet~ - logdet) / 2 and
    # g~ - g = (tr~ - tr) / 2 (the paper's NLL and gradient equations).
    assert es["loss"] - ex["loss"] == pytest.approx(0.5 * (es["logdet"] - ex["logdet"]),
                                                    abs=1e-9 * abs(ex["loss"]))
    np.testing.assert_allclose(es["grad"] - ex["grad"], 0.5 * (es["trace"] - ex["trace"]),
                               atol=1e-9 * np.abs(ex["grad"]).max())


# ------------------------------------------- per-dimension length-scales --

@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_ard_equal_lengthscales_reduce_to_isotropic(kind):
    X = inputs.points(60, 3, seed=41)
    y = inputs.gaussian_block(60, 1, seed=42)[:, 0].astype(np.float64)
    s, f, l = 0.2, 1.1, 0.35
    np.testing.assert_allclose(O.kernel_ard(X, X, kind, [l] * 3),
                               O.kernel_value(O.sqdist(X, X), kind, l), rtol=1e-12, atol=1e-15)
    iso = O.exact_nll(X, y, kind, (s, f, l))
    ard = O.exact_nll_ard(X, y, kind, s, f, [l] * 3)
    assert ard["loss"] == pytest.approx(iso["loss"], rel=1e-12)
    # d/dl of the isotropic loss is the sum of the per-dimension derivatives.
    np.testing.assert_allclose(ard["grad"][:2], iso["grad"][:2], rtol=1e-10)
    assert ard["grad"][2:].sum() == pytest.approx(iso["grad"][2], rel=1e-10)


def test_ard_gaussian_is_a_product_over_dimensions():
    rng = np.random.default_rng(43)
    A, B = rng.random((7, 4)), rng.random((5, 4))
    ls = [0.2, 0.5, 1.3, 0.05]
    prod = np.ones((7, 5))
    for t in range(4):
        prod *= np.exp(-(A[:, t][:, None] - B[:, t][None, :]) ** 2 / (2 * ls[t] ** 2))
    np.testing.assert_allclose(O.kernel_ard(A, B, O.GAUSSIAN, ls), prod, rtol=1e-13)


@pytest.mark.parametrize("kind,sampler", [(O.GAUSSIAN, _bochner_gaussian),
                                          (O.MATERN32, _bochner_matern32)])
def test_ard_kernel_matches_spectral_representation(kind, sampler):
    # Scaling coordinate t by 1/l_t maps the ARD kernel onto the unit isotropic
    # one, whose spectral measure is sampled independently of the formulas.
    rng = np.random.default_rng(44)
    ls = np.array([0.4, 1.1, 0.7])
    for delta in (np.array([0.3, 0.0, 0.0]), np.array([0.1, 0.5, -0.2]), np.array([0.0, 0.9, 0.4])):
        mc = sampler(delta / ls, 1.0, 400_000, rng)
        k = O.kernel_ard(delta[None, :], np.zeros((1, 3)), kind, ls)[0, 0]
        assert abs(mc - k) < 6e-3, (kind, delta, mc, k)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_ard_gradient_central_difference(kind):
    X = inputs.points(40, 3, seed=45)
    y = inputs.gaussian_block(40, 1, seed=46)[:, 0].astype(np.float64)
    s, f, ls = 0.15, 0.9, [0.3, 0.6, 0.45]
    g = O.exact_nll_ard(X, y, kind, s, f, ls)["grad"]
    params = [s, f] + list(ls)

    def L(p):
        return O.exact_nll_ard(X, y, kind, p[0], p[1], p[2:])["loss"]
    for t in range(len(params)):
        h = 1e-5 * params[t]
        up, dn = list(params), list(params)
        up[t] += h
        dn[t] -= h
        fd = (L(up) - L(dn)) / (2 * h)
        assert g[t] == pytest.approx(fd, rel=1e-6, abs=1e-8), (t, g[t], fd)


def test_est_nll_ard_approaches_exact():
    X = inputs.points(200, 2, seed=47)
    y = inputs.gaussian_block(200, 1, seed=48)[:, 0].astype(np.float64)
    s, f, ls = 0.1, 1.0, [0.15, 0.4]
    ex = O.exact_nll_ard(X, y, O.GAUSSIAN, s, f, ls)
    es = O.est_nll_ard(X, y, O.GAUSSIAN, s, f, ls, O.rademacher_probes(200, 256, 2), 30)
    np.testing.assert_allclose(es["quad"], ex["quad"], rtol=1e-12)
    assert es["loss"] - ex["loss"] == pytest.approx(0.5 * (es["logdet"] - ex["logdet"]),
                                                    abs=1e-9 * abs(ex["loss"]))
    # 256 probes: the estimated traces are within a few percent of the exact ones.
    assert np.all(np.abs(es["trace"] - ex["trace"]) <= 0.05 * np.abs(ex["trace"]) + 1.0)


# -------------------------------------------------------------------- CG --

def test_cg_matches_cholesky_solve():
    X = inputs.points(200, 3, seed=15)
    A = O.khat_dense(X, O.GAUSSIAN, (0.1, 1.0, 0.3))
    B = inputs.gaussian_block(200, 3, seed=5).astype(np.float64)
    Xs, iters, relres, _, _ = O.cg(A, B, 1e-10, 1000)
    ref = sla.cho_solve(sla.cho_factor(A), B)
    kappa = np.linalg.cond(A)
    assert np.all(relres <= 1e-10)
    for c in range(3):
        err = np.linalg.norm(Xs[:, c] - ref[:, c]) / np.linalg.norm(ref[:, c])
        assert err <= kappa * 1e-10 * 10
    assert np.all(iters < 200)


def test_cg_maxit_reports_residual():
    X = inputs.points(200, 2, seed=16)
    A = O.khat_dense(X, O.GAUSSIAN, (1e-3, 1.0, 0.3))
    b = np.ones(200)
    _, iters, relres, _, _ = O.cg(A, b, 1e-14, 3)
    assert iters[0] == 3 and relres[0] > 1e-14


# -------------------------------------------------- pivoted Cholesky, PCG --

def test_pivoted_cholesky_full_rank_is_a_permuted_cholesky():
    prob = inputs.small_problem(seed=21, n=120)
    A = prob.theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, prob.theta[2])
    A += 1e-6 * np.eye(120)
    L, piv, d = O.pivoted_cholesky(A, 120)
    assert sorted(piv.tolist()) == list(range(120))
    np.testing.assert_allclose(L @ L.T, A, rtol=0, atol=1e-11 * np.abs(A).max())
    # The factor restricted to the pivot rows is the (lower) Cholesky factor of
    # the permuted matrix, computed independently by LAPACK.
    P = A[np.ix_(piv, piv)]
    np.testing.assert_allclose(L[piv, :], sla.cholesky(P, lower=True), rtol=0, atol=1e-9)
    assert np.all(np.abs(d) <= 1e-10)


def test_pivoted_cholesky_greedy_rule_and_trace():
    rng = np.random.default_rng(22)
    G = rng.standard_normal((40, 40))
    A = G @ G.T + 40 * np.eye(40)
    L, piv, d = O.pivoted_cholesky(A, 10)
    # The first pivot is the largest diagonal entry; the residual diagonal is
    # diag(A - L L^T), and the residual trace never grows.
    assert piv[0] == int(np.argmax(np.diag(A)))
    np.testing.assert_allclose(d, np.diag(A - L @ L.T), atol=1e-9)
    traces = [np.trace(A - L[:, :j] @ L[:, :j].T) for j in range(11)]
    assert all(b <= a + 1e-9 for a, b in zip(traces, traces[1:]))
    # Each pivot is the argmax of the residual diagonal before its step.
    for j in range(10):
        dj = np.diag(A - L[:, :j] @ L[:, :j].T)
        assert piv[j] == int(np.argmax(dj))


def test_pivoted_cholesky_on_given_pivots_interpolates_their_columns():
    # Any pivot sequence: L L^T reproduces A on the pivot columns (the Nystrom
    # interpolation property) and L restricted to the pivot rows is lower
    # triangular; the greedy sequence given back reproduces the greedy factor.
    prob = inputs.small_problem(seed=26, n=150)
    A = prob.theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, prob.theta[2])
    piv = np.random.default_rng(27).permutation(150)[:12]
    L, got, _ = O.pivoted_cholesky(A, 12, pivots=piv)
    assert got.tolist() == piv.tolist()
    np.testing.assert_allclose((L @ L.T)[:, piv], A[:, piv], rtol=0, atol=1e-12)
    assert np.allclose(np.triu(L[piv, :], 1), 0.0)
    L0, p0, d0 = O.pivoted_cholesky(A, 12)
    L1, p1, d1 = O.pivoted_cholesky(A, 12, pivots=p0)
    assert p1.tolist() == p0.tolist()
    np.testing.assert_array_equal(L1, L0)
    np.testing.assert_array_equal(d1, d0)


def test_pivoted_cholesky_stops_at_the_exact_rank():
    # Points in 3 identical clusters: f^2 K has rank 3 (Gaussian, distinct
    # cluster centres), so the greedy factor stops after 3 steps.
    X = np.repeat(np.array([[0.1, 0.2], [0.7, 0.4], [0.3, 0.9]]), 20, axis=0)
    A = O.kernel_value(O.sqdist(X, X), O.GAUSSIAN, 0.3)
    L, piv, d = O.pivoted_cholesky(A, 10, tol=1e-10)
    assert L.shape[1] == 3
    np.testing.assert_allclose(L @ L.T, A, atol=1e-10)


def test_nystrom_woodbury_inverse_matches_dense_solve():
    rng = np.random.default_rng(23)
    L = rng.standard_normal((60, 7))
    V = rng.standard_normal((60, 3))
    s = 0.3
    got = O.nystrom_apply_inverse(L, s, V)
    ref = np.linalg.solve(L @ L.T + s * np.eye(60), V)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_pcg_with_the_matrix_itself_converges_in_one_step():
    prob = inputs.small_problem(seed=24, n=200)
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    b = prob.y.astype(np.float64)
    X, it, rel = O.pcg(Kh, b, lambda V: np.linalg.solve(Kh, V), 1e-10, 50)
    assert it[0] == 1 and rel[0] <= 1e-10
    np.testing.assert_allclose(X[:, 0], sla.cho_solve(sla.cho_factor(Kh), b), rtol=1e-8)


def test_pcg_with_identity_is_cg_and_nystrom_needs_fewer_iterations():
    prob = inputs.precision_problem(seed=25, n=1500)
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    b = prob.y.astype(np.float64)
    s, f, l = prob.theta
    X0, it0, _, _, _ = O.cg(Kh, b, 1e-8, 5000)
    X1, it1, _ = O.pcg(Kh, b, lambda V: V, 1e-8, 5000)
    assert it1[0] == it0[0]
    np.testing.assert_allclose(X1, X0, rtol=1e-10, atol=1e-10 * np.abs(X0).max())
    A = f * f * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, l)
    # About 500 eigenvalues of f^2 K exceed s here; a rank-600 Nystrom factor
    # takes most of the spectrum above s out of the iteration.
    L, _, _ = O.pivoted_cholesky(A, 600)
    X2, it2, rel2 = O.pcg(Kh, b, lambda V: O.nystrom_apply_inverse(L, s, V), 1e-8, 5000)
    assert rel2[0] <= 1e-8 and it2[0] < it0[0] / 5
    ref = sla.cho_solve(sla.cho_factor(Kh), b)
    assert np.linalg.norm(X2[:, 0] - ref) <= 1e-5 * np.linalg.norm(ref)


# ---------------------------------------------- pins catch planted mistakes --

def test_planted_sign_error_in_dl_is_caught(monkeypatch):
    good = O.kernel_dl
    monkeypatch.setattr(O.gp_oracle, "kernel_dl", lambda r2, kind, l: -good(r2, kind, l))
    with pytest.raises(AssertionError):
        test_exact_grad_central_difference(O.GAUSSIAN)


def test_planted_dropped_noise_term_is_caught(monkeypatch):
    monkeypatch.setattr(O.gp_oracle, "khat_dense",
                        lambda X, kind, th: th[1] ** 2 * O.kernel_value(O.sqdist(X, X), kind, th[2]))
    with pytest.raises(Exception):
        test_exact_nll_far_points_closed_form(O.GAUSSIAN)


def test_planted_transposed_cross_product_is_caught(monkeypatch):
    # A cross product taking points in the wrong order changes the shape/values.
    orig = O.gp_oracle.sqdist
    monkeypatch.setattr(O.gp_oracle, "sqdist", lambda A, B: orig(B, A).T * 1.0001)
    with pytest.raises(AssertionError):
        test_kmv_rows_brute_force(O.GAUSSIAN)


def test_planted_first_column_quadrature_is_caught(monkeypatch):
    # Weights from the first column of the eigenvector matrix instead of the first row.
    def wrong(a, b, znorm2):
        if a.size == 1:
            return znorm2 * math.log(a[0])
        lam, U = sla.eigh_tridiagonal(a, b)
        return znorm2 * float(np.sum(U[:, 0] ** 2 * np.log(lam)))
    monkeypatch.setattr(O.gp_oracle, "gauss_quadrature_log", wrong)
    monkeypatch.setattr(O, "gauss_quadrature_log", wrong)
    with pytest.raises(AssertionError):
        test_lanczos_full_length_equals_matrix_log()


def test_planted_normalised_probes_in_slq_are_caught(monkeypatch):
    # ||z||^2 dropped from the SLQ value (probes taken as unit vectors).
    good = O.gp_oracle.gauss_quadrature_log
    monkeypatch.setattr(O.gp_oracle, "gauss_quadrature_log", lambda a, b, z2: good(a, b, 1.0))
    with pytest.raises(AssertionError):
        test_slq_converges_to_logdet_within_3_sigma()


def test_planted_trace_sign_in_estimated_gradient_is_caught(monkeypatch):
    orig_est = O.gp_oracle.est_nll
    def est_wrong(X, y, kind, theta, Z, k):
        out = orig_est(X, y, kind, theta, Z, k)
        out["grad"] = 0.5 * (-out["quad"] - out["trace"])
        return out
    monkeypatch.setattr(O.gp_oracle, "est_nll", est_wrong)
    monkeypatch.setattr(O, "est_nll", est_wrong)
    with pytest.raises(AssertionError):
        test_est_nll_approaches_exact()


def test_planted_noisy_variance_is_caught(monkeypatch):
    # Adding the noise s (the variance of a noisy observation) to the
    # noise-free predictive variance.
    good = O.gp_oracle.predict_var
    monkeypatch.setattr(O, "predict_var", lambda X, Xs, k, th: good(X, Xs, k, th) + th[0])
    with pytest.raises(AssertionError):
        test_predict_var_far_points_is_the_prior(O.GAUSSIAN)


def test_planted_unscaled_cross_covariance_is_caught(monkeypatch):
    # k_c = K(X, x*) without the f^2 scale: the quadratic term shrinks by f^4.
    good = O.gp_oracle.predict_var
    def wrong(X, Xs, k, th):
        f2 = th[1] ** 2
        return f2 - (f2 - good(X, Xs, k, th)) / (f2 * f2)
    monkeypatch.setattr(O, "predict_var", wrong)
    with pytest.raises(AssertionError):
        test_predict_var_identical_points_closed_form(O.GAUSSIAN)


def test_planted_wrong_ard_derivative_power_is_caught(monkeypatch):
    # dK/dl_t with l_t^2 in place of l_t^3.
    good = O.gp_oracle.kernel_dls
    def wrong(A, B, kind, ls):
        return [D * ls[t] for t, D in enumerate(good(A, B, kind, ls))]
    monkeypatch.setattr(O.gp_oracle, "kernel_dls", wrong)
    with pytest.raises(AssertionError):
        test_ard_gradient_central_difference(O.GAUSSIAN)


def test_planted_wrong_woodbury_sign_is_caught(monkeypatch):
    good = O.gp_oracle.nystrom_apply_inverse
    def wrong(L, s, V):
        return 2.0 * V / s - good(L, s, V)
    monkeypatch.setattr(O, "nystrom_apply_inverse", wrong)
    with pytest.raises(AssertionError):
        test_nystrom_woodbury_inverse_matches_dense_solve()


# ------------------------------------- Eq. 1 / Eq. 2 with a Nystrom M --

def _precond_case(n=60, seed=41, kind=1, theta=(0.05, 1.2, 0.3)):
    prob = inputs.uniform_problem(n, 3, kind, theta, seed=seed)
    return prob, prob.theta


def test_nystrom_precond_derivatives_match_central_differences():
    prob, theta = _precond_case()
    A = theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, theta[2])
    _, piv, _ = O.pivoted_cholesky(A, 8)
    M, dMs = O.nystrom_precond(prob.X, prob.kind, theta, piv)
    for t in range(3):
        h = 1e-5 * theta[t]
        tp = list(theta); tp[t] += h
        tm = list(theta); tm[t] -= h
        Mp, _ = O.nystrom_precond(prob.X, prob.kind, tp, piv)
        Mm, _ = O.nystrom_precond(prob.X, prob.kind, tm, piv)
        fd = (Mp - Mm) / (2 * h)
        np.testing.assert_allclose(dMs[t], fd, rtol=0, atol=1e-6 * np.abs(fd).max() + 1e-12)


def test_nystrom_precond_logdet_by_the_determinant_identity():
    # |s I_n + L L^T| = s^(n-r) |s I_r + L^T L| (Sylvester), with L the partial
    # Cholesky factor on the same pivots (L L^T = B W^-1 B^T).
    prob, theta = _precond_case()
    s = theta[0]
    A = theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, theta[2])
    L, piv, _ = O.pivoted_cholesky(A, 10)
    M, _ = O.nystrom_precond(prob.X, prob.kind, theta, piv)
    n, r = L.shape
    ref = (n - r) * math.log(s) + np.linalg.slogdet(s * np.eye(r) + L.T @ L)[1]
    assert abs(np.linalg.slogdet(M)[1] - ref) <= 1e-9 * abs(ref)
    np.testing.assert_allclose(M, s * np.eye(n) + L @ L.T, atol=1e-12)


def test_precond_estimator_is_exact_when_m_is_kh():
    # Every point a pivot: M = Kh, so log|M| = log|Kh|, M^-1/2 Kh M^-1/2 = I
    # (its SLQ term is log 1 = 0 for any probe) and each Hutchinson term is
    # zero: the estimator is the exact loss and gradient whatever the probes.
    prob, theta = _precond_case(n=50)
    A = theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, theta[2])
    _, piv, _ = O.pivoted_cholesky(A, 50)
    rng = np.random.default_rng(42)
    est = O.est_nll_precond(prob.X, prob.y, prob.kind, theta, piv, rng.standard_normal((50, 3)),
                            rng.standard_normal((50, 3)), 4)
    ex = O.exact_nll(prob.X, prob.y, prob.kind, theta)
    assert abs(est["loss"] - ex["loss"]) <= 1e-8 * abs(ex["loss"])
    np.testing.assert_allclose(est["grad"], ex["grad"], rtol=1e-7, atol=1e-9)
    assert np.abs(est["logdet_probes"]).max() <= 1e-9
    assert np.abs(est["trace_corr"]).max() <= 1e-7


def test_precond_slq_term_is_exact_at_full_krylov_dimension():
    prob, theta = _precond_case(n=40)
    A = theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, theta[2])
    _, piv, _ = O.pivoted_cholesky(A, 6)
    rng = np.random.default_rng(43)
    E1, E2 = rng.standard_normal((6, 2)), rng.standard_normal((40, 2))
    est = O.est_nll_precond(prob.X, prob.y, prob.kind, theta, piv, E1, E2, 40)
    M, _ = O.nystrom_precond(prob.X, prob.kind, theta, piv)
    lam, U = np.linalg.eigh(M)
    Mis = (U / np.sqrt(lam)) @ U.T
    Ah = Mis @ O.khat_dense(prob.X, prob.kind, theta) @ Mis
    la, Ua = np.linalg.eigh(Ah)
    logA = (Ua * np.log(la)) @ Ua.T
    Zh = Mis @ est["Z"]
    ref = np.array([Zh[:, i] @ logA @ Zh[:, i] for i in range(2)])
    np.testing.assert_allclose(est["logdet_probes"], ref, rtol=1e-8)


def test_precond_trace_estimator_is_unbiased_with_lower_variance():
    # z ~ N(0, M): the mean of the Eq. 2 terms converges to tr(Kh^-1 dKh).  When
    # the factor covers the eigenvalues of f^2 K above s (16 here; rank 25), the
    # split off tr(M^-1 dM) leaves a far smaller variance than Gaussian probes
    # with M = I (z ~ N(0, I), tr ~ (Kh^-1 z)^T dKh z).
    prob = inputs.uniform_problem(120, 2, O.GAUSSIAN, (0.02, 1.0, 0.4), seed=41)
    theta = prob.theta
    A = theta[1] ** 2 * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, theta[2])
    _, piv, _ = O.pivoted_cholesky(A, 25)
    rng = np.random.default_rng(44)
    p = 1500
    est = O.est_nll_precond(prob.X, prob.y, prob.kind, theta, piv, rng.standard_normal((25, p)),
                            rng.standard_normal((120, p)), 3)
    Kh = O.khat_dense(prob.X, prob.kind, theta)
    dKs = O.dkhat_dense(prob.X, prob.kind, theta)
    exact_tr = np.array([np.trace(np.linalg.solve(Kh, dK)) for dK in dKs])
    vals = est["trace_M"][:, None] + est["trace_corr"]
    se = vals.std(axis=1, ddof=1) / math.sqrt(p)
    assert np.all(np.abs(vals.mean(axis=1) - exact_tr) <= 4 * se + 1e-12)
    G = rng.standard_normal((120, p))
    plain = np.array([np.sum(np.linalg.solve(Kh, G) * (dK @ G), axis=0) for dK in dKs])
    assert np.all(vals.std(axis=1) < 0.2 * plain.std(axis=1))


def test_gaussian_probes_are_standard_normal():
    G = O.gaussian_probes(4000, 2, seed=7)
    assert abs(G.mean()) <= 4 / math.sqrt(G.size)
    assert abs(G.var() - 1.0) <= 4 * math.sqrt(2.0 / G.size)
    from scipy import stats
    assert stats.kstest(G.ravel(), "norm").pvalue > 1e-3
    # Columns and seeds give different streams; rows are not shifted copies.
    assert not np.allclose(G[:, 0], G[:, 1])
    assert not np.allclose(O.gaussian_probes(50, 1, 8)[:, 0], G[:50, 0])
    assert not np.allclose(G[1:51, 0], G[:50, 0])


def test_planted_mistakes_in_the_preconditioned_estimator_are_caught(monkeypatch):
    good = O.gp_oracle.nystrom_precond

    def wrong_sign(X, kind, theta, piv):
        M, d = good(X, kind, theta, piv)
        return M, [d[0], d[1], -d[2]]
    monkeypatch.setattr(O.gp_oracle, "nystrom_precond", wrong_sign)
    monkeypatch.setattr(O, "nystrom_precond", wrong_sign)
    with pytest.raises(AssertionError):
        test_nystrom_precond_derivatives_match_central_differences()
    with pytest.raises(AssertionError):
        test_precond_estimator_is_exact_when_m_is_kh()
