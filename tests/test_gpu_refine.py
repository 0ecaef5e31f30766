"""Mixed-precision iterative refinement: tensor-core inner CG, compensated
FP32-pair outer residual (or FP64 on request).

Bounds:
 - after refinement the true residual ||B - Kh X||_2 / ||B||_2 of the FP64
   solution, recomputed here by the FP64 oracle, is <= 1e-6; the FP32-output
   form is additionally limited by the rounding of X to FP32 (about
   u ||Kh|| ||X|| / ||B||);
 - the residual rows themselves (gp_residual_rows) agree with the dense FP64
   oracle's B - Kh X to 1e-9 ||B_c|| per column in the pair arithmetic and
   1e-12 ||B_c|| in FP64, at a near-solution X (where B - Kh X cancels most).
"""
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


# Refinement converges when kappa * (relative product error) < 1: BF16 (~5e-3) at
# kappa ~ 6e2 (s = 1), TF32 (~3e-4) and split BF16 (~1e-5) also at kappa ~ 6e3.
# Outer residual 0 = FP32 pair (the default), 1 = FP64.
@pytest.mark.parametrize("prec,s_noise,resid", [(1, 1.0, 0), (2, 1.0, 0), (1, 0.1, 0), (4, 0.1, 0),
                                                (3, 0.1, 0), (4, 0.1, 1)])
def test_refinement_reaches_1e6_true_residual(api, prec, s_noise, resid):
    prob = inputs.small_problem(seed=3)
    theta = (s_noise, prob.theta[1], prob.theta[2])
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 3, seed=4)]).astype(np.float32)
    opts = api.solve_opts(cg_rtol=1e-2, prec=prec, refine_rtol=1e-7, refine_maxit=30,
                          refine_residual=resid)
    Xs, iters, relres, st = api.gp_pcg_solve_refined(_dev(prob.X), _dev(Bm), prob.kind, theta, opts)
    assert st == 0 and max(relres) <= 1e-7
    Kh = O.khat_dense(prob.X, prob.kind, theta)
    Xg = Xs.cpu().numpy()
    true_res = np.linalg.norm(Bm - Kh @ Xg, axis=0) / np.linalg.norm(Bm, axis=0)
    assert true_res.max() <= 1e-6, true_res
    # The FP32-output form agrees up to the rounding of X.
    X32, _, rel32, st32 = api.gp_pcg_solve(_dev(prob.X), _dev(Bm), prob.kind, theta, opts)
    assert st32 == 0
    assert np.abs(X32.cpu().numpy() - Xg).max() <= 1e-6 * np.abs(Xg).max()
    ref = sla.cho_solve(sla.cho_factor(Kh), Bm.astype(np.float64))
    err = np.linalg.norm(Xg - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= np.linalg.cond(Kh) * 1e-6


def test_refinement_reports_not_converged(api):
    prob = inputs.small_problem(seed=4)
    opts = api.solve_opts(cg_rtol=1e-1, prec=1, refine_rtol=1e-12, refine_maxit=1)
    _, iters, relres, st = api.gp_pcg_solve(_dev(prob.X), _dev(prob.y), prob.kind, prob.theta, opts,
                                            raise_not_converged=False)
    assert st == 4 and relres[0] > 1e-12 and iters[0] > 0


def test_refinement_beats_fp32_cg_true_residual(api):
    # Plain FP32 CG plateaus near u * kappa; refinement reaches 1e-6.
    prob = inputs.small_problem(seed=5)
    X, y = _dev(prob.X), _dev(prob.y)
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    x32, _, _, _ = api.gp_pcg_solve(X, y, prob.kind, prob.theta, api.solve_opts(cg_rtol=1e-10),
                                   raise_not_converged=False)
    xr, _, _, _ = api.gp_pcg_solve_refined(X, y, prob.kind, prob.theta,
                                           api.solve_opts(cg_rtol=1e-2, prec=4, refine_rtol=1e-7,
                                                          refine_maxit=30))
    yy = prob.y.astype(np.float64)
    r32 = np.linalg.norm(yy - Kh @ x32.cpu().numpy()[:, 0].astype(np.float64)) / np.linalg.norm(yy)
    rr = np.linalg.norm(yy - Kh @ xr.cpu().numpy()[:, 0]) / np.linalg.norm(yy)
    assert rr <= 1e-6 and rr < r32


def test_true_residual_matches_oracle(api):
    # gp_true_residual (FP64 entries and sums) against the dense FP64 oracle on
    # the FP32 CG solution of three columns.
    prob = inputs.small_problem(seed=6)
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 2, seed=8)]).astype(np.float32)
    Xs, _, _, _ = api.gp_pcg_solve(_dev(prob.X), _dev(Bm), prob.kind, prob.theta,
                                   api.solve_opts(cg_rtol=1e-6), raise_not_converged=False)
    rel = api.gp_true_residual(_dev(prob.X), _dev(Bm), Xs, prob.kind, prob.theta)
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    Xh = Xs.cpu().numpy().astype(np.float64)
    ref = np.linalg.norm(Bm - Kh @ Xh, axis=0) / np.linalg.norm(Bm, axis=0)
    np.testing.assert_allclose(rel, ref, rtol=1e-6, atol=0)


def test_workspace_contents_are_ignored(api):
    # Every call treats its workspace as scratch: a workspace full of NaN bytes
    # gives the same results as a fresh one.
    import torch
    from paper_2503_02259_gb300 import _binding as B
    prob = inputs.small_problem(seed=7)
    X, y = _dev(prob.X), _dev(prob.y)
    V = _dev(inputs.multivector(prob.y, 11, seed=1))
    pr, _ = api.problem(X, prob.kind, prob.theta)

    def poisoned(op, w, opts=None):
        ws = api.workspace(op, pr, w, opts, X.device)
        ws.fill_(0xFF)
        return ws

    Y0 = api.gp_kernel_matmul(X, V, prob.kind, prob.theta)
    Y1 = api.gp_kernel_matmul(X, V, prob.kind, prob.theta, ws=poisoned(B.OP_MATMUL, 11))
    assert torch.equal(Y0, Y1)
    for prec in (3, 4):
        o = api.solve_opts(prec=prec)
        Y0 = api.gp_kernel_matmul(X, V, prob.kind, prob.theta, prec=prec)
        Y1 = api.gp_kernel_matmul(X, V, prob.kind, prob.theta, prec=prec,
                                  ws=poisoned(B.OP_MATMUL, 11, o))
        assert torch.equal(Y0, Y1)
    G0 = api.gp_kernel_grad_matmul(X, V, prob.kind, prob.theta)
    G1 = api.gp_kernel_grad_matmul(X, V, prob.kind, prob.theta, ws=poisoned(B.OP_GRAD_MATMUL, 11))
    for a, b in zip(G0, G1):
        assert torch.equal(a, b)
    xs, _, _, _ = api.gp_pcg_solve(X, y, prob.kind, prob.theta, api.solve_opts(cg_rtol=1e-6),
                                   raise_not_converged=False)
    r0 = api.gp_true_residual(X, y, xs, prob.kind, prob.theta)
    r1 = api.gp_true_residual(X, y, xs, prob.kind, prob.theta, ws=poisoned(B.OP_RESIDUAL, 1))
    assert r0 == r1 and r0[0] < 1e-3
    # Solvers: CG (FP32 and a refined tensor-core solve), SLQ, loss + gradient, prediction.
    o = api.solve_opts(cg_rtol=1e-6)
    a0 = api.gp_pcg_solve(X, y, prob.kind, prob.theta, o)
    a1 = api.gp_pcg_solve(X, y, prob.kind, prob.theta, o, ws=poisoned(B.OP_PCG, 1, o))
    assert torch.equal(a0[0], a1[0]) and a0[1:] == a1[1:]
    o = api.solve_opts(cg_rtol=1e-2, prec=4, refine_rtol=1e-7, refine_maxit=30)
    b0 = api.gp_pcg_solve_refined(X, y, prob.kind, prob.theta, o)
    b1 = api.gp_pcg_solve_refined(X, y, prob.kind, prob.theta, o, ws=poisoned(B.OP_PCG, 1, o))
    assert torch.equal(b0[0], b1[0]) and b0[1:] == b1[1:]
    o = api.solve_opts(nprobe=6, nlanczos=20, seed=3, prec=4, slq_prec=3)
    assert (api.gp_slq_logdet(X, prob.kind, prob.theta, o) ==
            api.gp_slq_logdet(X, prob.kind, prob.theta, o, ws=poisoned(B.OP_SLQ, 0, o)))
    o = api.solve_opts(nprobe=6, nlanczos=20, seed=3, cg_rtol=1e-6)
    l0 = api.gp_loss_and_grad(X, y, prob.kind, prob.theta, o)
    l1 = api.gp_loss_and_grad(X, y, prob.kind, prob.theta, o, ws=poisoned(B.OP_LOSS_GRAD, 0, o))
    assert l0[0] == l1[0] and l0[1] == l1[1]
    Xs = _dev(inputs.points(300, 3, seed=9))
    m0 = api.gp_predict_mean(X, a0[0][:, 0].contiguous(), Xs, prob.kind, prob.theta)
    m1 = api.gp_predict_mean(X, a0[0][:, 0].contiguous(), Xs, prob.kind, prob.theta,
                             ws=poisoned(B.OP_PREDICT, 300))
    assert torch.equal(m0, m1)


def _oracle_residual(X, Bm, X64, kind, theta):
    Kh = O.khat_dense(X, kind, theta)
    return Bm.astype(np.float64) - Kh @ X64


@pytest.mark.parametrize("n,d,kind,theta,w", [
    (2000, 3, 0, (0.1, 1.0, 0.3), 3),       # the small problem
    (1037, 2, 0, (0.01, 1.0, 0.05), 1),     # the precision problem's kernel, ragged n
    (1500, 3, 1, (0.05, 1.5, 0.2), 6),      # the fused matvec problem's kernel
    (777, 8, 0, (0.1, 1.0, 1.2), 4),        # d = 8 (the differentiation problem's kernel)
    (300, 16, 1, (0.2, 0.7, 0.9), 9),       # d = 16, two column groups of 8
    (129, 1, 1, (0.3, 1.2, 0.4), 2),        # d = 1, one row past a block
])
def test_residual_rows_match_dense_oracle_near_solution(api, n, d, kind, theta, w):
    import scipy.linalg as sla
    X = inputs.points(n, d, seed=n + d)
    Bm = inputs.gaussian_block(n, w, seed=11).astype(np.float32)
    Kh = O.khat_dense(X, kind, theta)
    X64 = sla.cho_solve(sla.cho_factor(Kh), Bm.astype(np.float64))   # near-solution: cancellation
    ref = _oracle_residual(X, Bm, X64, kind, theta)
    bn = np.linalg.norm(Bm.astype(np.float64), axis=0)
    for arith, tol in ((0, 1e-9), (1, 1e-12)):
        R, rel = api.gp_residual_rows(_dev(X), _dev(Bm), _dev(X64), kind, theta, arith=arith)
        Rh = R.cpu().numpy()
        err = np.linalg.norm(Rh - ref, axis=0) / bn
        assert err.max() <= tol, (arith, err)
        np.testing.assert_allclose(rel, np.linalg.norm(Rh, axis=0) / bn, rtol=1e-12)
    # A far-from-solution X: the residual is O(||B||) and agrees to the same bounds.
    Xr = inputs.gaussian_block(n, w, seed=12).astype(np.float64)
    ref = _oracle_residual(X, Bm, Xr, kind, theta)
    for arith, tol in ((0, 1e-9), (1, 1e-12)):
        R, _ = api.gp_residual_rows(_dev(X), _dev(Bm), _dev(Xr), kind, theta, arith=arith)
        assert (np.linalg.norm(R.cpu().numpy() - ref, axis=0) / bn).max() <= tol


def test_residual_rows_on_sampled_rows(api):
    import torch
    prob = inputs.small_problem(seed=9)
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 1, seed=2)]).astype(np.float32)
    X64 = inputs.gaussian_block(prob.n, 2, seed=3).astype(np.float64)
    ref = _oracle_residual(prob.X, Bm, X64, prob.kind, prob.theta)
    rows = np.random.default_rng(4).choice(prob.n, 333, replace=False)
    rows_d = torch.from_numpy(rows.astype(np.int64)).cuda()
    for arith, tol in ((0, 1e-9), (1, 1e-12)):
        R, rel = api.gp_residual_rows(_dev(prob.X), _dev(Bm), _dev(X64), prob.kind, prob.theta,
                                      rows=rows_d, arith=arith)
        Rh = R.cpu().numpy()
        scale = np.linalg.norm(Bm[rows].astype(np.float64), axis=0)
        assert (np.linalg.norm(Rh - ref[rows], axis=0) / scale).max() <= tol
        np.testing.assert_allclose(rel, np.linalg.norm(Rh, axis=0) / scale, rtol=1e-12)
    # The first m rows when no index array is given.
    R, _ = api.gp_residual_rows(_dev(prob.X), _dev(Bm), _dev(X64), prob.kind, prob.theta, m=200)
    assert R.shape == (200, 2)
    assert np.abs(R.cpu().numpy() - ref[:200]).max() <= 1e-9 * np.abs(ref).max()


def test_residual_rows_rejects_out_of_range_indices(api):
    import torch
    from paper_2503_02259_gb300 import _binding as B
    prob = inputs.small_problem(seed=10)
    X64 = torch.zeros((prob.n, 1), dtype=torch.float64, device="cuda")
    rows = torch.tensor([0, 5, prob.n, 7], dtype=torch.int64, device="cuda")
    with pytest.raises(B.GPError) as ei:
        api.gp_residual_rows(_dev(prob.X), _dev(prob.y), X64, prob.kind, prob.theta, rows=rows)
    assert ei.value.status == B.GP_ERR_ARG
    # The library stays usable.
    R, rel = api.gp_residual_rows(_dev(prob.X), _dev(prob.y), X64, prob.kind, prob.theta,
                                  rows=rows[:2])
    np.testing.assert_allclose(R.cpu().numpy()[:, 0], prob.y[[0, 5]], rtol=0, atol=0)


def test_pair_and_fp64_refinement_agree(api):
    # The same refinement with either outer residual reaches the target, and the
    # solutions agree to the refinement tolerance.
    prob = inputs.small_problem(seed=12)
    X, y = _dev(prob.X), _dev(prob.y)
    out = []
    for resid in (0, 1):
        o = api.solve_opts(cg_rtol=1e-2, prec=4, refine_rtol=1e-8, refine_maxit=30,
                           refine_residual=resid)
        xr, _, rr, st = api.gp_pcg_solve_refined(X, y, prob.kind, prob.theta, o)
        assert st == 0 and rr[0] <= 1e-8
        out.append(xr.cpu().numpy()[:, 0])
    Kh = O.khat_dense(prob.X, prob.kind, prob.theta)
    yy = prob.y.astype(np.float64)
    for x in out:
        assert np.linalg.norm(yy - Kh @ x) / np.linalg.norm(yy) <= 1e-7
