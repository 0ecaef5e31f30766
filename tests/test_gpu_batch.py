"""Batched loss and gradient (gp_loss_and_grad_batch): several problems, one
grouped product launch per solver step.

Bounds: each member's loss and gradient equal its own gp_loss_and_grad result
bit for bit when the batch keeps the member's padded width (the grouped kernel
evaluates the same entries in the same order, and the O(n w) steps are the
same launches), and within 1e-9 relative otherwise (a padded width changes
only the order of the FP64 reductions); each member also matches the FP64
oracle's same-probe estimator at the 1e-4 loss / gradient bound.
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


def _members(d, kind, count, seed0):
    rng = np.random.default_rng(seed0)
    out = []
    for k in range(count):
        n = int(rng.integers(300, 3000))
        theta = (float(rng.uniform(0.05, 0.3)), float(rng.uniform(0.7, 1.5)),
                 float(rng.uniform(0.15, 0.5)))
        out.append(inputs.uniform_problem(n, d, kind, theta, seed=seed0 + k))
    return out


@pytest.mark.parametrize("d,kind,nprobe,exact", [(3, O.GAUSSIAN, 10, True),   # w = 11 -> 12
                                                 (2, O.MATERN32, 16, True),   # w = 17 -> 20
                                                 (8, O.GAUSSIAN, 6, False)])  # w = 7 -> 12
def test_batch_equals_one_at_a_time(env, d, kind, nprobe, exact):
    torch, B, api = env
    probs = _members(d, kind, 6, seed0=10 * d + nprobe)
    opts = [api.solve_opts(nprobe=nprobe, nlanczos=15, cg_rtol=1e-7, seed=3 + k)
            for k in range(len(probs))]
    Xs = [_dev(p.X) for p in probs]
    ys = [_dev(p.y) for p in probs]
    losses, grads, infos, status = api.gp_loss_and_grad_batch(
        Xs, ys, [p.kind for p in probs], [p.theta for p in probs], opts)
    assert all(s == 0 for s in status)
    for k, p in enumerate(probs):
        l1, g1, i1 = api.gp_loss_and_grad(Xs[k], ys[k], p.kind, p.theta, opts[k])
        if exact:
            assert losses[k] == l1 and grads[k] == g1 and infos[k]["cg_iters"] == i1["cg_iters"]
        else:
            assert losses[k] == pytest.approx(l1, rel=1e-9)
            np.testing.assert_allclose(grads[k], g1, rtol=1e-9, atol=1e-9 * np.abs(g1).max())


def test_batch_matches_oracle_and_respects_each_cap(env):
    torch, B, api = env
    probs = _members(3, O.MATERN32, 4, seed0=77)
    nprobe, k = 8, 20
    opts = [api.solve_opts(nprobe=nprobe, nlanczos=k, cg_rtol=1e-8, seed=5 + j)
            for j in range(len(probs))]
    opts.append(api.solve_opts(nprobe=nprobe, nlanczos=k, cg_rtol=1e-12, cg_maxit=7, seed=1))
    probs.append(inputs.uniform_problem(1500, 3, O.MATERN32, (0.01, 1.0, 0.4), seed=99))
    Xs = [_dev(p.X) for p in probs]
    ys = [_dev(p.y) for p in probs]
    losses, grads, infos, status = api.gp_loss_and_grad_batch(
        Xs, ys, [p.kind for p in probs], [p.theta for p in probs], opts, raise_not_converged=False)
    assert status[:-1] == [0] * (len(probs) - 1) and status[-1] == B.GP_ERR_NOT_CONVERGED
    assert infos[-1]["cg_iters"] == 7
    for j, p in enumerate(probs[:-1]):
        est = O.est_nll(p.X, p.y, p.kind, p.theta, O.rademacher_probes(p.n, nprobe, 5 + j), k)
        assert abs(losses[j] - est["loss"]) <= 1e-4 * abs(est["loss"])
        g = np.asarray(est["grad"])
        floor = 1e-3 * np.linalg.norm(g)
        for t in range(3):
            assert abs(grads[j][t] - g[t]) <= 1e-4 * max(abs(g[t]), floor)


def test_batch_rejects_mixed_templates(env):
    torch, B, api = env
    a = inputs.uniform_problem(500, 3, O.GAUSSIAN, (0.1, 1.0, 0.3), seed=1)
    b = inputs.uniform_problem(500, 8, O.GAUSSIAN, (0.1, 1.0, 0.3), seed=2)
    o = api.solve_opts(nprobe=4, nlanczos=10)
    with pytest.raises(B.GPError) as ei:
        api.gp_loss_and_grad_batch([_dev(a.X), _dev(b.X)], [_dev(a.y), _dev(b.y)],
                                   [a.kind, b.kind], [a.theta, b.theta], [o, o])
    assert ei.value.status == B.GP_ERR_ARG


@pytest.mark.parametrize("count", [1, 64])
def test_batch_sizes_one_and_the_maximum(env, count):
    torch, B, api = env
    rng = np.random.default_rng(count)
    probs = [inputs.uniform_problem(int(rng.integers(129, 400)), 2, O.MATERN32,
                                    (0.2, 1.0, float(rng.uniform(0.2, 0.5))), seed=500 + k)
             for k in range(count)]
    opts = [api.solve_opts(nprobe=4, nlanczos=10, cg_rtol=1e-6, seed=k) for k in range(count)]
    Xs = [_dev(p.X) for p in probs]
    ys = [_dev(p.y) for p in probs]
    losses, grads, _, status = api.gp_loss_and_grad_batch(
        Xs, ys, [p.kind for p in probs], [p.theta for p in probs], opts)
    assert status == [0] * count
    for k in (0, count // 2, count - 1):
        l1, g1, _ = api.gp_loss_and_grad(Xs[k], ys[k], probs[k].kind, probs[k].theta, opts[k])
        assert losses[k] == pytest.approx(l1, rel=1e-9)
        np.testing.assert_allclose(grads[k], g1, rtol=1e-9, atol=1e-9 * np.abs(g1).max())
    if count == 64:
        with pytest.raises(B.GPError) as ei:
            api.gp_loss_and_grad_batch(Xs + Xs[:1], ys + ys[:1], [probs[0].kind] * 65,
                                       [p.theta for p in probs] + [probs[0].theta], opts + opts[:1])
        assert ei.value.status == B.GP_ERR_ARG
