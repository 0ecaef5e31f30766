"""Nystrom-preconditioned CG: the pivoted partial Cholesky factor, M^-1 V by the
Woodbury identity, and the preconditioned solves (plain and refined).

Bounds, from the arithmetic:
 - the factor: the GPU stores each column in FP32 and computes the next one
   exactly for the stored columns (pair kernel entry, Dot2 sums), so column j
   differs from the FP64 oracle's (on the same pivots) by the propagated
   storage rounding, a few u f^2 / sqrt(d_{p_j}) (u = 2^-24), checked with a
   factor 64 of slack; a pivot is valid when its oracle residual diagonal is
   within 64 u f^2 of the largest, and must equal the oracle's argmax when the
   top two are further apart than that;
 - M^-1 V: exact for the stored factor up to the final rounding to FP32 and
   the FP64 inverse of C (kappa(C) 2^-53): 1e-6 of ||M^-1 V_c|| per column;
 - solves: the FP32 true-residual floor u ||Kh|| ||x|| / ||b|| (times 64) on
   top of cg_rtol; refined solves: 1e-6 recomputed by the FP64 oracle.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2503_02259_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


def _fK(prob, theta=None):
    s, f, l = prob.theta if theta is None else theta
    return f * f * O.kernel_value(O.sqdist(prob.X, prob.X), prob.kind, l)


def _check_pivots(A, piv, f2):
    """Each GPU pivot is an argmax of the oracle's residual diagonal on the
    GPU's earlier pivots (exactly the argmax where it is unique to 64 u f^2)."""
    tol = 64 * U32 * f2
    L, _, _ = O.pivoted_cholesky(A, len(piv), pivots=piv)
    assert piv[0] == 0
    for j, p in enumerate(piv):
        dj = np.diag(A) - np.sum(L[:, :j] ** 2, axis=1)
        dj[np.asarray(piv[:j], dtype=int)] = -np.inf
        order = np.argsort(-dj, kind="stable")
        assert dj[p] >= dj[order[0]] - tol, (j, p, dj[p], dj[order[0]])
        if dj[order[0]] - dj[order[1]] > 2 * tol:
            assert p == order[0], (j, p, order[0])
    return L


@pytest.mark.parametrize("kind,n,k,w", [(0, 701, 60, 5), (1, 1000, 120, 1), (0, 257, 16, 8)])
def test_factor_and_apply_match_the_oracle(api, kind, n, k, w):
    prob = inputs.uniform_problem(n, 3, kind, (0.1, 1.3, 0.3), seed=31)
    V = inputs.gaussian_block(n, w, seed=32).astype(np.float32)
    Z, Lg, piv, rank = api.gp_nystrom_apply(_dev(prob.X), _dev(V), kind, prob.theta, k, want_L=True)
    assert rank == k and len(piv) == k
    A = _fK(prob)
    f2 = prob.theta[1] ** 2
    Lo = _check_pivots(A, piv, f2)
    Lg = Lg.cpu().numpy().astype(np.float64)
    for j in range(k):
        dp = Lo[piv[j], j] ** 2
        err = np.abs(Lg[:, j] - Lo[:, j]).max()
        assert err <= 64 * U32 * (f2 / np.sqrt(dp) + np.abs(Lo[:, j]).max()), (j, err, dp)
    # M^-1 V for the stored factor, by the oracle's Woodbury solve (itself
    # pinned against a dense solve).
    ref = O.nystrom_apply_inverse(Lg, prob.theta[0], V.astype(np.float64))
    Zg = Z.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(Zg - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 1e-6, rel


def test_rank_one_factor_is_the_first_kernel_column(api):
    prob = inputs.uniform_problem(300, 2, 1, (0.05, 0.7, 0.2), seed=33)
    V = np.ones((300, 1), dtype=np.float32)
    _, Lg, piv, rank = api.gp_nystrom_apply(_dev(prob.X), _dev(V), 1, prob.theta, 1, want_L=True)
    assert rank == 1 and piv == [0]
    col = _fK(prob)[:, 0] / prob.theta[1]
    np.testing.assert_allclose(Lg.cpu().numpy()[:, 0], col, rtol=4 * U32, atol=4 * U32)


def test_exact_rank_stops_the_factor(api):
    # Three clusters of identical points: f^2 K has rank 3 (Gaussian kernel,
    # distinct centres), so the factor stops after three pivots, one per cluster.
    X = np.repeat(np.array([[0.1, 0.2], [0.7, 0.4], [0.3, 0.9]], dtype=np.float32), 40, axis=0)
    V = inputs.gaussian_block(120, 2, seed=34).astype(np.float32)
    theta = (0.2, 1.0, 0.3)
    Z, Lg, piv, rank = api.gp_nystrom_apply(_dev(X), _dev(V), 0, theta, 10, tol=1e-5, want_L=True)
    assert rank == 3
    assert sorted(p // 40 for p in piv) == [0, 1, 2]
    Lg = Lg.cpu().numpy().astype(np.float64)
    A = O.kernel_value(O.sqdist(X, X), O.GAUSSIAN, 0.3)
    np.testing.assert_allclose(Lg @ Lg.T, A, atol=1e-6)
    ref = np.linalg.solve(theta[0] * np.eye(120) + Lg @ Lg.T, V.astype(np.float64))
    Zg = Z.cpu().numpy()
    assert np.linalg.norm(Zg - ref) <= 1e-6 * np.linalg.norm(ref)


def _true_relres(Kh, Bm, Xg):
    return np.linalg.norm(Bm - Kh @ Xg, axis=0) / np.linalg.norm(Bm, axis=0)


def _fp32_floor(Kh, Bm, Xg):
    nK = np.linalg.norm(Kh, 2)
    return 64 * U32 * nK * np.linalg.norm(Xg, axis=0) / np.linalg.norm(Bm, axis=0)


def test_preconditioned_cg_matches_the_oracle_and_cuts_iterations(api):
    # The oracle's pinned case: n = 1500 points of the precision problem's
    # kernel (d = 2, Gaussian l = 0.05, s = 0.01), rank 600.
    prob = inputs.precision_problem(seed=25, n=1500)
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 2, seed=35)]).astype(np.float32)
    rtol = 1e-5
    opts = api.solve_opts(cg_rtol=rtol, cg_maxit=5000, precond_rank=600)
    Xs, it, rel, st = api.gp_pcg_solve(_dev(prob.X), _dev(Bm), prob.kind, prob.theta, opts)
    assert st == 0 and max(rel) <= rtol
    opts0 = api.solve_opts(cg_rtol=rtol, cg_maxit=5000)
    _, it0, _, st0 = api.gp_pcg_solve(_dev(prob.X), _dev(Bm), prob.kind, prob.theta, opts0)
    assert st0 == 0
    assert max(it) * 5 < min(it0), (it, it0)
    # The oracle's PCG with the GPU's own factor takes about as many steps.
    _, Lg, _, rank = api.gp_nystrom_apply(_dev(prob.X), _dev(Bm[:, :1]), prob.kind, prob.theta, 600,
                                          want_L=True)
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    Lg = Lg.cpu().numpy().astype(np.float64)
    _, ito, _ = O.pcg(Kh, Bm.astype(np.float64),
                      lambda V: O.nystrom_apply_inverse(Lg, prob.theta[0], V), rtol, 5000)
    assert np.all(np.abs(np.asarray(it) - ito) <= 2), (it, ito)
    Xg = Xs.cpu().numpy().astype(np.float64)
    tr = _true_relres(Kh, Bm.astype(np.float64), Xg)
    assert np.all(tr <= 2 * rtol + _fp32_floor(Kh, Bm, Xg)), tr


def test_full_rank_preconditioner_solves_in_a_few_steps(api):
    # k >= n: M = s I + L L^T reproduces Kh up to the factor's rounding.
    prob = inputs.uniform_problem(300, 3, 1, (0.1, 1.0, 0.4), seed=36)
    opts = api.solve_opts(cg_rtol=1e-6, cg_maxit=300, precond_rank=4096)
    Xs, it, rel, st = api.gp_pcg_solve(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    assert st == 0 and it[0] <= 4, it
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    ref = sla.cho_solve(sla.cho_factor(Kh), prob.y.astype(np.float64))
    assert np.linalg.norm(Xs.cpu().numpy()[:, 0] - ref) <= 1e-4 * np.linalg.norm(ref)


def test_preconditioner_with_per_dimension_length_scales(api):
    prob = inputs.uniform_problem(1200, 3, 0, (0.01, 1.0, 1.0), seed=37)
    ls = [0.15, 0.3, 0.6]
    rtol = 1e-5
    opts = api.solve_opts(cg_rtol=rtol, cg_maxit=5000, precond_rank=300)
    Xs, it, rel, st = api.gp_pcg_solve(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts, ls=ls)
    assert st == 0
    _, it0, _, _ = api.gp_pcg_solve(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta,
                                    api.solve_opts(cg_rtol=rtol, cg_maxit=5000), ls=ls)
    assert it[0] * 3 < it0[0], (it, it0)
    Kh = O.khat_dense_ard(prob.X, prob.kind, prob.theta[0], prob.theta[1], np.asarray(ls))
    Xg = Xs.cpu().numpy().astype(np.float64)
    y = prob.y.astype(np.float64)[:, None]
    assert _true_relres(Kh, y, Xg)[0] <= 2 * rtol + _fp32_floor(Kh, y, Xg)[0]


@pytest.mark.parametrize("prec", [0, 4])
def test_refinement_with_the_preconditioner_reaches_1e6(api, prec):
    # kappa ~ 1e5: n = 3000 points of the precision problem's kernel.
    prob = inputs.precision_problem(seed=38, n=3000)
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 1, seed=39)]).astype(np.float32)
    opts = api.solve_opts(cg_rtol=1e-3, cg_maxit=2000, prec=prec, refine_rtol=1e-7, refine_maxit=20,
                          precond_rank=900)
    X64, it, rel, st = api.gp_pcg_solve_refined(_dev(prob.X), _dev(Bm), prob.kind, prob.theta, opts)
    assert st == 0 and max(rel) <= 1e-7
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    tr = _true_relres(Kh, Bm.astype(np.float64), X64.cpu().numpy())
    assert tr.max() <= 1e-6, tr
    opts0 = api.solve_opts(cg_rtol=1e-3, cg_maxit=5000, prec=prec, refine_rtol=1e-7,
                           refine_maxit=20)
    _, it0, rel0, st0 = api.gp_pcg_solve_refined(_dev(prob.X), _dev(Bm), prob.kind, prob.theta, opts0)
    assert st0 == 0
    assert max(it) * 5 < min(it0), (it, it0)


# ------------------------------------- the loss with the preconditioner --
# Eq. 1 / Eq. 2 with M = s I + L L^T (pivots fixed).  Bounds: log|M| to 1e-7
# relative (FP64 Cholesky of the exact-sum Gram of the stored factor against
# the oracle's dense slogdet); tr(M^-1 dM) to 1e-5 relative (dL/dl stored in
# FP32); loss and gradient to the 1e-4 bound of the unpreconditioned
# estimator, against the oracle's estimator on the same pivots and normal values.

def _loss_precond(api, prob, rank, p, k, eps=None, tol=0.0, seed=0):
    # opts holds only the probe block's address: keep the tensor alive for the call.
    eps_d = None if eps is None else _dev(eps)
    opts = api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-8, cg_maxit=5000, precond_rank=rank,
                          precond_tol=tol, probes=eps_d, seed=seed)
    out = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    del eps_d
    return out


def _pivots(api, prob, rank, tol):
    _, _, piv, _ = api.gp_nystrom_apply(_dev(prob.X), _dev(prob.y[:, None]), prob.kind, prob.theta,
                                        rank, tol=tol)
    return piv


def _check_loss(loss, grad, ref_loss, ref_grad):
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss), (loss, ref_loss)
    g = np.asarray(grad)
    scale = np.maximum(np.abs(ref_grad), 1e-3 * np.linalg.norm(ref_grad))
    assert np.all(np.abs(g - ref_grad) / scale <= 1e-4), (g, ref_grad)


@pytest.mark.parametrize("kind,n,d,theta,rank,tol", [
    (0, 600, 2, (0.05, 1.0, 0.4), 80, 1e-6),
    (1, 500, 3, (0.05, 1.2, 0.5), 120, 1e-5),
])
def test_preconditioned_loss_matches_the_oracle(api, kind, n, d, theta, rank, tol):
    prob = inputs.uniform_problem(n, d, kind, theta, seed=51)
    p, k = 8, 25
    eps = np.random.default_rng(52).standard_normal((n + rank, p)).astype(np.float32)
    loss, grad, info = _loss_precond(api, prob, rank, p, k, eps=eps, tol=tol)
    piv = _pivots(api, prob, rank, tol)
    r = len(piv)
    est = O.est_nll_precond(prob.X, prob.y, prob.kind, prob.theta, piv,
                            eps[n:n + r].astype(np.float64), eps[:n].astype(np.float64), k)
    assert abs(info["logdet_m"] - est["logdet_M"]) <= 1e-7 * abs(est["logdet_M"])
    np.testing.assert_allclose(info["trace_m"], est["trace_M"], rtol=1e-5)
    _check_loss(loss, grad, est["loss"], est["grad"])


@pytest.mark.parametrize("prec,slq", [(4, 3), (3, 3)])
def test_preconditioned_loss_in_split_tensor_core_arithmetic(api, prec, slq):
    # Split BF16 CG with split TF32 Lanczos, and split TF32 throughout: the
    # solves and Lanczos products run on the tensor cores, the preconditioner and
    # the derivative product in FP32.  A product entry carries at most ~4.3e-6
    # relative error in either arithmetic, so to first order the solves and the
    # loss may move by kappa(Kh) times that: the bound below.
    n, d, rank, p, k = 700, 2, 100, 8, 25
    prob = inputs.uniform_problem(n, d, 0, (0.05, 1.0, 0.2), seed=51)
    ev = np.linalg.eigvalsh(O.khat_dense(prob.X, prob.kind, prob.theta))
    tol = max(1e-4, ev[-1] / ev[0] * 4.3e-6)
    eps = np.random.default_rng(54).standard_normal((n + rank, p)).astype(np.float32)
    eps_d = _dev(eps)
    opts = api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-8, cg_maxit=5000, precond_rank=rank,
                          probes=eps_d, prec=prec, slq_prec=slq)
    loss, grad, info = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    piv = _pivots(api, prob, rank, 0.0)
    est = O.est_nll_precond(prob.X, prob.y, prob.kind, prob.theta, piv,
                            eps[n:n + len(piv)].astype(np.float64), eps[:n].astype(np.float64), k)
    # log|M| comes from the FP32 factor alone, whatever the product arithmetic.
    assert abs(info["logdet_m"] - est["logdet_M"]) <= 1e-7 * abs(est["logdet_M"])
    assert abs(loss - est["loss"]) <= tol * abs(est["loss"]), (loss, est["loss"], tol)
    g, gr = np.asarray(grad), est["grad"]
    scale = np.maximum(np.abs(gr), 1e-3 * np.linalg.norm(gr))
    assert np.all(np.abs(g - gr) / scale <= tol), (g, gr, tol)


def test_preconditioned_loss_with_every_point_a_pivot_is_exact(api):
    # M = Kh up to the factor's rounding: the stochastic terms vanish for any
    # probes (generated on the device here) and the estimate is the exact loss.
    prob = inputs.uniform_problem(250, 3, 1, (0.05, 1.0, 0.3), seed=53)
    loss, grad, info = _loss_precond(api, prob, 4096, 4, 10, seed=3)
    ex = O.exact_nll(prob.X, prob.y, prob.kind, prob.theta)
    _check_loss(loss, grad, ex["loss"], ex["grad"])


def test_generated_gaussian_probes_match_the_oracle_generator(api):
    prob = inputs.uniform_problem(300, 2, 0, (0.05, 1.0, 0.4), seed=54)
    rank, p, k, seed, tol = 40, 4, 15, 11, 1e-6
    loss, grad, _ = _loss_precond(api, prob, rank, p, k, tol=tol, seed=seed)
    piv = _pivots(api, prob, rank, tol)
    r = len(piv)
    G = O.gaussian_probes(300 + r, p, seed)
    est = O.est_nll_precond(prob.X, prob.y, prob.kind, prob.theta, piv, G[300:300 + r], G[:300], k)
    _check_loss(loss, grad, est["loss"], est["grad"])


def test_preconditioned_estimator_has_a_smaller_spread(api):
    # With the spectrum above s covered by the factor, Eq. 1 / Eq. 2's split
    # leaves stochastic terms with a far smaller spread than M = I, and the
    # solves take fewer iterations.
    prob = inputs.uniform_problem(600, 2, 0, (0.05, 1.0, 0.4), seed=51)
    _, _, ip = _loss_precond(api, prob, 80, 16, 25, tol=1e-6, seed=5)
    opts = api.solve_opts(nprobe=16, nlanczos=25, cg_rtol=1e-8, cg_maxit=5000, seed=5)
    _, _, i0 = api.gp_loss_and_grad(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts)
    assert ip["logdet_stderr"] < i0["logdet_stderr"] / 3, (ip["logdet_stderr"], i0["logdet_stderr"])
    for t in range(3):
        assert ip["trace_stderr"][t] < i0["trace_stderr"][t] / 3, (t, ip["trace_stderr"], i0["trace_stderr"])
    assert ip["cg_iters"] < i0["cg_iters"]


def test_autograd_wrapper_takes_the_preconditioner(api):
    import torch
    from paper_2503_02259_gb300 import autograd
    prob = inputs.uniform_problem(400, 2, 0, (0.05, 1.0, 0.4), seed=55)
    theta = torch.tensor(prob.theta, dtype=torch.float64, requires_grad=True)
    X, y = _dev(prob.X), _dev(prob.y)
    L = autograd.neg_log_likelihood(theta, X, y, prob.kind, nprobe=8, nlanczos=20, cg_rtol=1e-8,
                                    seed=9, precond_rank=60, precond_tol=1e-6)
    (g,) = torch.autograd.grad(2.0 * L, theta)
    opts = api.solve_opts(nprobe=8, nlanczos=20, cg_rtol=1e-8, seed=9, precond_rank=60,
                          precond_tol=1e-6)
    loss, grad, _ = api.gp_loss_and_grad(X, y, prob.kind, prob.theta, opts)
    assert float(L) == loss
    np.testing.assert_array_equal(g.numpy(), 2.0 * np.asarray(grad))
