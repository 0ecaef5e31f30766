"""Mixed-precision iterative refinement: tensor-core inner CG, FP64 outer residual.

Bound (mixed-precision path): after refinement the true residual
||B - Kh X||_2 / ||B||_2 of the FP64 solution, recomputed here by the FP64
oracle, is <= 1e-6.  The FP32-output form is additionally limited by the
rounding of X to FP32 (about u ||Kh|| ||X|| / ||B||).
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
@pytest.mark.parametrize("prec,s_noise", [(1, 1.0), (2, 1.0), (1, 0.1), (4, 0.1), (3, 0.1)])
def test_refinement_reaches_1e6_true_residual(api, prec, s_noise):
    prob = inputs.small_problem(seed=3)
    theta = (s_noise, prob.theta[1], prob.theta[2])
    Bm = np.column_stack([prob.y, inputs.gaussian_block(prob.n, 3, seed=4)]).astype(np.float32)
    opts = api.solve_opts(cg_rtol=1e-2, prec=prec, refine_rtol=1e-7, refine_maxit=30)
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
