"""Per-dimension length-scales (ARD) on the GPU against the FP64 oracle.

Bounds: products at the FP32 bound 1e-5 (norm-wise per column; split BF16
3e-5); the loss and each of the 2 + d gradient components against the
oracle's same-probe estimator at |delta| / max(|ref|, 1e-3 ||g_ref||) <= 1e-4,
as for the isotropic loss.  With equal length-scales the ARD path (a fused
contraction of the entries with alpha alpha^T and U Z^T / p) and the isotropic
path (a derivative product) must agree: the loss bit for bit (the same staged
points), s to 1e-12 (the same terms, reduced in another order), and f and the
sum of the l_t components at the 1e-4
gradient bound (the f component is a difference of two terms some 100 times
larger, so the two FP32 summation orders already differ by ~3e-5 of it).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_02259_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import _binding as B
    from paper_2503_02259_gb300 import api
    return torch, B, api


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


@pytest.mark.parametrize("n,d,kind,ls,w", [
    (1500, 3, O.GAUSSIAN, [0.2, 0.5, 1.1], 11),
    (1031, 2, O.MATERN32, [0.05, 0.3], 32),
    (700, 8, O.GAUSSIAN, [0.6, 0.9, 1.3, 2.0, 0.8, 1.0, 1.7, 0.5], 5),
    (300, 16, O.MATERN32, list(np.linspace(0.4, 2.5, 16)), 17),
])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (4, 3e-5)])
def test_ard_products_match_oracle(env, n, d, kind, ls, w, prec, tol):
    torch, B, api = env
    s, f = 0.1, 1.2
    X = inputs.points(n, d, seed=n + d)
    V = inputs.gaussian_block(n, w, seed=w)
    Y = api.gp_kernel_matmul(_dev(X), _dev(V), kind, (s, f, 1.0), prec=prec, ls=ls).cpu().numpy()
    ref = f * f * (O.kernel_ard(X, X, kind, ls) @ V.astype(np.float64)) + s * V
    assert _relerr(Y, ref) <= tol


CASES = [
    (1200, 2, O.GAUSSIAN, 0.1, 1.0, [0.15, 0.4]),
    (1500, 3, O.MATERN32, 0.05, 1.5, [0.2, 0.35, 0.5]),
    (900, 8, O.GAUSSIAN, 0.1, 1.0, [1.0, 1.5, 0.8, 1.2, 2.0, 0.9, 1.1, 1.4]),
]


@pytest.mark.parametrize("n,d,kind,s,f,ls", CASES)
def test_ard_loss_and_gradient_match_oracle_estimator(env, n, d, kind, s, f, ls):
    torch, B, api = env
    X = inputs.points(n, d, seed=2 * n + d)
    y = (np.sin(4 * X[:, 0]) + X[:, -1]).astype(np.float32)
    p, k, seed = 8, 25, 11
    opts = api.solve_opts(nprobe=p, nlanczos=k, cg_rtol=1e-8, seed=seed)
    loss, grad, info = api.gp_loss_and_grad(_dev(X), _dev(y), kind, (s, f, 1.0), opts, ls=ls)
    est = O.est_nll_ard(X, y, kind, s, f, ls, O.rademacher_probes(n, p, seed), k)
    assert len(grad) == 2 + d
    assert abs(loss - est["loss"]) <= 1e-4 * abs(est["loss"])
    g = np.asarray(est["grad"])
    floor = 1e-3 * np.linalg.norm(g)
    for t in range(2 + d):
        assert abs(grad[t] - g[t]) <= 1e-4 * max(abs(g[t]), floor), (t, grad, g)
    assert np.isnan(info["quad"][2]) and info["quad"][0] == pytest.approx(est["quad"][0], rel=1e-4)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_ard_with_equal_lengthscales_is_the_isotropic_path(env, kind):
    torch, B, api = env
    prob = inputs.small_problem(seed=2)
    theta = prob.theta if kind == O.GAUSSIAN else (0.05, 1.5, 0.2)
    opts = api.solve_opts(nprobe=6, nlanczos=20, cg_rtol=1e-8, seed=3)
    X, y = _dev(prob.X), _dev(prob.y)
    li, gi, _ = api.gp_loss_and_grad(X, y, kind, theta, opts)
    la, ga, _ = api.gp_loss_and_grad(X, y, kind, theta, opts, ls=[theta[2]] * 3)
    assert la == li and ga[0] == pytest.approx(gi[0], rel=1e-12)
    floor = 1e-3 * np.linalg.norm(gi)
    for a, b in ((ga[1], gi[1]), (sum(ga[2:]), gi[2])):
        assert abs(a - b) <= 1e-4 * max(abs(b), floor), (ga, gi)


def test_ard_prediction_mean(env):
    torch, B, api = env
    n, d, s, f, ls = 1000, 3, 0.1, 1.1, [0.2, 0.6, 0.35]
    X = inputs.points(n, d, seed=9)
    Xs = inputs.points(257, d, seed=10)
    alpha = inputs.gaussian_block(n, 1, seed=11)[:, 0]
    mu = api.gp_predict_mean(_dev(X), _dev(alpha), _dev(Xs), O.GAUSSIAN, (s, f, 1.0), ls=ls)
    ref = f * f * (O.kernel_ard(Xs, X, O.GAUSSIAN, ls) @ alpha.astype(np.float64))
    assert np.linalg.norm(mu.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5


def test_ard_unsupported_paths_say_so(env):
    torch, B, api = env
    prob = inputs.small_problem(seed=4, n=500)
    X, y = _dev(prob.X), _dev(prob.y)
    ls = [0.3, 0.4, 0.5]
    with pytest.raises(B.GPError) as ei:
        api.gp_pcg_solve(X, y, prob.kind, prob.theta,
                         api.solve_opts(prec=4, refine_rtol=1e-7, cg_rtol=1e-2), ls=ls)
    assert ei.value.status == B.GP_ERR_UNIMPLEMENTED
    pr, _ = api.problem(X, prob.kind, prob.theta, ls)
    V = _dev(inputs.gaussian_block(500, 4, seed=1))
    Y, dY = torch.empty_like(V), torch.empty_like(V)
    ws = api.workspace(B.OP_GRAD_MATMUL, pr, 4, None, X.device)
    st = B.lib().gp_kernel_grad_matmul(B.ctypes.byref(pr), api._ptr(V), 4, api._ptr(Y), None,
                                       api._ptr(dY), 0, api._ptr(ws), ws.numel(), api._stream(X.device))
    assert st == B.GP_ERR_UNIMPLEMENTED
    with pytest.raises(B.GPError) as ei:
        api.gp_loss_and_grad(X, y, prob.kind, prob.theta, api.solve_opts(nprobe=60, nlanczos=5),
                             ls=ls)
    assert ei.value.status == B.GP_ERR_UNIMPLEMENTED
    # Invalid length-scales are argument errors.
    with pytest.raises(B.GPError) as ei:
        api.gp_kernel_matmul(X, V, prob.kind, prob.theta, ls=[0.3, -1.0, 0.5])
    assert ei.value.status == B.GP_ERR_ARG


def test_ard_autograd_backward_matches_oracle(env):
    # The differentiable loss with theta = (s, f, l_1..l_d): one backward gives
    # all 2 + d components, equal to the oracle's same-probe estimator.
    torch, B, api = env
    from paper_2503_02259_gb300.autograd import neg_log_likelihood
    n, d, kind, s, f, ls = 1000, 3, O.GAUSSIAN, 0.1, 1.2, [0.25, 0.4, 0.6]
    X = inputs.points(n, d, seed=61)
    y = (np.cos(3 * X[:, 1]) + X[:, 0]).astype(np.float32)
    theta = torch.tensor([s, f] + ls, dtype=torch.float64, requires_grad=True)
    for recompute in (False, True):
        L = neg_log_likelihood(theta, _dev(X), _dev(y), kind, nprobe=8, nlanczos=25, cg_rtol=1e-8,
                               seed=13, recompute=recompute)
        (g,) = torch.autograd.grad(L, theta)
        est = O.est_nll_ard(X, y, kind, s, f, ls, O.rademacher_probes(n, 8, 13), 25)
        assert abs(L.item() - est["loss"]) <= 1e-4 * abs(est["loss"])
        gr = np.asarray(est["grad"])
        floor = 1e-3 * np.linalg.norm(gr)
        assert np.all(np.abs(g.numpy() - gr) <= 1e-4 * np.maximum(np.abs(gr), floor)), (g, gr)
