"""GPU parity of block CG, SLQ, Hutchinson and L(Theta) / dL/dTheta against the
FP64 oracle, through the C ABI.

Tolerances:
  * loss and each gradient component vs the oracle's same-probe estimator
    (O-est): |delta| / max(|ref|, 1e-3 ||g_ref||) <= 1e-4;
  * vs the exact Cholesky values (O-exact): y^T alpha and the quadratic
    gradient terms at 1e-4; log-det and traces within 4 standard errors of the
    probe mean (they are stochastic estimates);
  * CG: recurrence relres <= cg_rtol; true residual checked in FP64.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2503_02259_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import api as A
    return A


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b, floor=0.0):
    return abs(a - b) / max(abs(b), floor, 1e-300)


@pytest.fixture(scope="module")
def small():
    prob = inputs.small_problem(seed=0)
    Z = O.rademacher_probes(prob.n, 10, 1234)
    est = O.est_nll(prob.X, prob.y, prob.kind, prob.theta, Z, 30)
    ex = O.exact_nll(prob.X, prob.y, prob.kind, prob.theta)
    return prob, est, ex


@pytest.mark.parametrize("s_noise,true_tol", [(1.0, 2e-5), (0.1, 3e-4)])
def test_pcg_matches_cholesky(api, s_noise, true_tol):
    # The recurrence relres reaches cg_rtol; the true residual of an FP32-product
    # CG is bounded near u * kappa (u ~ 1e-7 the product's relative accuracy):
    # kappa ~ 6e2 at s = 1 and ~ 6e3 at s = 0.1 for this problem.
    prob = inputs.small_problem(seed=1)
    theta = (s_noise, prob.theta[1], prob.theta[2])
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 4, seed=3)]).astype(np.float32)
    opts = api.solve_opts(cg_rtol=1e-8)
    Xs, iters, relres, st = api.gp_pcg_solve(_dev(prob.X), _dev(Bm), prob.kind, theta, opts)
    assert st == 0
    assert max(relres) <= 1e-8
    Kh = O.khat_dense(prob.X, prob.kind, theta)
    Xg = Xs.cpu().numpy().astype(np.float64)
    true_res = np.linalg.norm(Bm - Kh @ Xg, axis=0) / np.linalg.norm(Bm, axis=0)
    assert true_res.max() <= true_tol, true_res
    ref = sla.cho_solve(sla.cho_factor(Kh), Bm.astype(np.float64))
    err = np.linalg.norm(Xg - ref, axis=0) / np.linalg.norm(ref, axis=0)
    kappa = np.linalg.cond(Kh)
    assert err.max() <= kappa * true_res.max(), (err, kappa)
    # FP64 CG with the same start and stopping rule needs no more iterations; the
    # FP32 recurrences lose orthogonality and converge later, but within 2x here.
    _, it_ref, _, _, _ = O.cg(Kh, Bm, 1e-8, 5000)
    assert np.all(np.array(iters) >= it_ref - 2) and np.all(np.array(iters) <= 2 * it_ref), (iters, it_ref)


def test_pcg_reports_not_converged(api):
    prob = inputs.small_problem(seed=2)
    opts = api.solve_opts(cg_rtol=1e-12, cg_maxit=5)
    _, iters, relres, st = api.gp_pcg_solve(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts,
                                            raise_not_converged=False)
    assert st == 4  # GP_ERR_NOT_CONVERGED
    assert iters == [5] and relres[0] > 1e-12


def test_slq_matches_same_probe_estimator(api, small):
    prob, est, ex = small
    opts = api.solve_opts(nprobe=10, nlanczos=30, cg_rtol=1e-10, seed=1234)
    ld, se = api.gp_slq_logdet(_dev(prob.X), prob.kind, prob.theta, opts)
    assert rel(ld, est["logdet"]) <= 1e-4, (ld, est["logdet"])
    assert abs(ld - ex["logdet"]) <= 4 * se + 1e-4 * abs(ex["logdet"])


def test_loss_and_grad_small_config(api, small):
    prob, est, ex = small
    opts = api.solve_opts(nprobe=10, nlanczos=30, cg_rtol=1e-8, seed=1234)
    loss, grad, info = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    gref = est["grad"]
    gfloor = 1e-3 * np.linalg.norm(gref)
    assert rel(loss, est["loss"]) <= 1e-4, (loss, est["loss"])
    for t in range(3):
        assert rel(grad[t], gref[t], gfloor) <= 1e-4, (t, grad, gref)
    # Against the exact (Cholesky) values: deterministic terms tight, stochastic in band.
    assert rel(info["yalpha"], ex["yalpha"]) <= 1e-4
    for t in range(3):
        assert rel(info["quad"][t], ex["quad"][t], 1e-3 * np.abs(ex["quad"]).max()) <= 1e-4
        assert abs(info["trace"][t] - ex["trace"][t]) <= 4 * info["trace_stderr"][t] + 1e-6
    assert abs(info["logdet"] - ex["logdet"]) <= 4 * info["logdet_stderr"]
    assert info["relres_max"] <= 1e-8


def test_forward_backward_split_equals_fused(api, small):
    prob, est, _ = small
    opts = api.solve_opts(nprobe=10, nlanczos=30, cg_rtol=1e-8, seed=1234)
    X, y = _dev(prob.X), _dev(prob.y)
    loss, grad, _ = api.gp_loss_and_grad(X, y, prob.kind, prob.theta, opts)
    loss2, W, _ = api.gp_nll_forward(X, y, prob.kind, prob.theta, opts)
    grad2, _ = api.gp_nll_backward(X, W, prob.kind, prob.theta, opts)
    assert loss2 == loss
    np.testing.assert_allclose(grad2, grad, rtol=1e-12, atol=0)


# (CG arithmetic, SLQ arithmetic) of the forward: FP32, and the mixed pair.
@pytest.mark.parametrize("prec,slq", [(0, 0), (4, 3)])
def test_autograd_function(api, small, prec, slq):
    import torch
    from paper_2503_02259_gb300.autograd import neg_log_likelihood
    prob, est, _ = small
    X, y = _dev(prob.X), _dev(prob.y)
    for recompute in (False, True):
        theta = torch.tensor(prob.theta, dtype=torch.float64, requires_grad=True)
        L = neg_log_likelihood(theta, X, y, prob.kind, nprobe=10, nlanczos=30, cg_rtol=1e-8,
                               seed=1234, recompute=recompute, prec=prec, slq_prec=slq)
        (2.0 * L).backward()
        g = theta.grad.numpy() / 2.0
        gfloor = 1e-3 * np.linalg.norm(est["grad"])
        for t in range(3):
            assert rel(g[t], est["grad"][t], gfloor) <= 1e-4
        assert rel(float(L.detach()), est["loss"]) <= 1e-4


@pytest.fixture(scope="module")
def diff_sub():
    # n = 4000 subsample of the d = 8, 0.5 N(0, I) differentiation problem;
    # Gaussian s = 0.1, f = 1, l = 1.2; 32 probes x 40 Lanczos steps.
    prob = inputs.diff_problem(seed=0, n=4000)
    Z = O.rademacher_probes(prob.n, 32, 77)
    return prob, O.est_nll(prob.X, prob.y, prob.kind, prob.theta, Z, 40)


# (CG arithmetic, SLQ arithmetic): FP32; split TF32 for both; split BF16 for the
# CG solves with split TF32 for the Lanczos products (the log-determinant needs
# ~24-bit kernel entries; split BF16 keeps 16).
@pytest.mark.parametrize("prec,slq", [(0, 0), (3, -1), (4, 3)])
def test_differentiation_config_subsample(api, diff_sub, prec, slq):
    prob, est = diff_sub
    opts = api.solve_opts(nprobe=32, nlanczos=40, cg_rtol=1e-8, seed=77, prec=prec, slq_prec=slq)
    loss, grad, info = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    gfloor = 1e-3 * np.linalg.norm(est["grad"])
    assert rel(loss, est["loss"]) <= 1e-4, (loss, est["loss"])
    for t in range(3):
        assert rel(grad[t], est["grad"][t], gfloor) <= 1e-4, (t, grad, est["grad"])


def test_loss_matern_and_user_probes(api):
    prob = inputs.uniform_problem(1500, 2, O.MATERN32, (0.05, 1.2, 0.25), seed=5)
    Z = O.rademacher_probes(prob.n, 8, 99).astype(np.float32)
    Zd = _dev(Z)
    est = O.est_nll(prob.X, prob.y, prob.kind, prob.theta, Z, 25)
    opts = api.solve_opts(nprobe=8, nlanczos=25, cg_rtol=1e-8, seed=0, probes=Zd)
    loss, grad, _ = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    gfloor = 1e-3 * np.linalg.norm(est["grad"])
    assert rel(loss, est["loss"]) <= 1e-4
    for t in range(3):
        assert rel(grad[t], est["grad"][t], gfloor) <= 1e-4


def test_slq_arithmetic_is_chosen_separately(api, small):
    # slq_prec selects the arithmetic of the Lanczos products alone: SLQ in FP32
    # under a tensor-core CG equals the all-FP32 log-determinant (up to the order
    # of the FP64 dot-product sums, which follows the padded width the two
    # products share), and GP_PREC_SAME equals naming the CG arithmetic.  A
    # tensor-core Lanczos product would move the result by ~1e-6.
    prob, est, ex = small
    X = _dev(prob.X)
    ld32, _ = api.gp_slq_logdet(X, prob.kind, prob.theta,
                                api.solve_opts(nprobe=10, nlanczos=30, seed=1234))
    ld_a, _ = api.gp_slq_logdet(X, prob.kind, prob.theta,
                                api.solve_opts(nprobe=10, nlanczos=30, seed=1234, prec=4, slq_prec=0))
    assert rel(ld_a, ld32) <= 1e-12
    ld_same, _ = api.gp_slq_logdet(X, prob.kind, prob.theta,
                                   api.solve_opts(nprobe=10, nlanczos=30, seed=1234, prec=3,
                                                  slq_prec=-1))
    ld_tf, _ = api.gp_slq_logdet(X, prob.kind, prob.theta,
                                 api.solve_opts(nprobe=10, nlanczos=30, seed=1234, prec=0, slq_prec=3))
    assert rel(ld_same, ld_tf) <= 1e-12
    assert rel(ld_tf, est["logdet"]) <= 1e-4


# The fused CG step (one cooperative launch with two grid barriers) against the
# three separate kernels it replaces: same sums in the same order, so the same
# bits.  Shapes: the small problem (w = 11, 63 reduction blocks), a ragged n,
# the largest reduction grid (608 blocks, all resident at once), a column
# that stops at maxit, and the split-TF32 product.
@pytest.mark.parametrize("n,w,prec,maxit", [(2000, 11, 0, 0), (1037, 5, 0, 0), (20000, 33, 0, 0),
                                            (3001, 17, 0, 7), (4096, 16, 3, 0)])
def test_fused_cg_step_equals_separate_kernels(api, monkeypatch, n, w, prec, maxit):
    import torch
    prob = inputs.uniform_problem(n, 3, 0, (0.05, 1.0, 0.2), seed=5)
    Bm = _dev(inputs.multivector(prob.y, w, seed=6))
    X = _dev(prob.X)
    opts = api.solve_opts(cg_rtol=1e-7, cg_maxit=maxit, prec=prec)
    runs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("GP_CG_FUSED", flag)
        Xs, iters, relres, st = api.gp_pcg_solve(X, Bm, prob.kind, prob.theta, opts,
                                                 raise_not_converged=False)
        torch.cuda.synchronize()
        runs.append((Xs.cpu(), iters, relres, st))
    (xa, ia, ra, sa), (xb, ib, rb, sb) = runs
    assert sa == sb and ia == ib and ra == rb
    assert torch.equal(xa, xb)
    if maxit:
        assert sa == 4 and max(ia) == maxit
    elif prec == 0:
        assert sa == 0 and max(ra) <= 1e-7


def test_fused_cg_step_loss_and_grad_bits(api, small, monkeypatch):
    prob, _, _ = small
    opts = api.solve_opts(nprobe=10, nlanczos=30, cg_rtol=1e-8, seed=1234)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("GP_CG_FUSED", flag)
        loss, grad, info = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
        out.append((loss, grad, info["cg_iters"]))
    assert out[0] == out[1]
