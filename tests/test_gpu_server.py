"""The continuous-batching server: each result is the same alone and in the mix,
admission respects the device-memory budget, oversize requests are refused.

Tolerances: results alone and in the mix are compared bit for bit, in FP32 and
in the mixed arithmetics the served form uses (every kernel is deterministic
and independent of what else runs); against the direct C calls likewise.
Served requests run to convergence (n <= 4000) are held to the FP64 oracle at
the loss / gradient bound 1e-4 (same probes, the oracle's estimator with exact
solves) and predictions to 1e-4 against the posterior mean from the exact
solution, on problems whose conditioning keeps the arithmetic's solution error
(about kappa times the product error) below that.
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
    from paper_2503_02259_gb300 import api, server
    return torch, api, server


def _requests():
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(8):
        n = int(rng.integers(400, 3000))
        d = [2, 3, 8][i % 3]
        kind = i % 2
        prob = inputs.uniform_problem(n, d, kind, (0.05 + 0.01 * i, 1.0 + 0.1 * i, 0.2 + 0.05 * i), seed=i)
        is_pred = (i % 4 == 3)
        Xs = inputs.points(300, d, seed=100 + i) if is_pred else None
        reqs.append((1 if is_pred else 0, prob, Xs))
    return reqs


def _run(server_mod, reqs, slots, budget=8 << 30, **kw):
    with server_mod.Server(budget, slots) as srv:
        tickets = []
        for kind, p, Xs in reqs:
            r, keep = server_mod.Server.request(kind, p.X, p.y, p.kind, p.theta, nprobe=6, Xstar=Xs,
                                                cg_maxit=400, nlanczos=15, cg_rtol=1e-6, seed=9, **kw)
            tickets.append(srv.submit(r, keep))
        srv.drain(300)
        out = [srv.poll(t) for t in tickets]
        return out, srv.stats()


# (CG arithmetic, SLQ arithmetic): FP32, split BF16 CG with split TF32 Lanczos
# (the served mixed form), split TF32 throughout.
ARITHMETICS = [(0, 0), (4, 3), (3, 3)]


@pytest.mark.parametrize("prec,slq", ARITHMETICS)
def test_results_same_alone_and_in_the_mix(env, prec, slq):
    torch, api, server = env
    reqs = _requests()
    alone = [_run(server, [r], 1, prec=prec, slq_prec=slq)[0][0] for r in reqs]
    mixed, stats = _run(server, reqs, 4, prec=prec, slq_prec=slq)
    assert stats["completed"] == len(reqs)
    assert stats["peak_active"] >= 2          # requests did share the device
    for a, b in zip(alone, mixed):
        assert a["status"] == b["status"]
        if a["mu"] is None:
            assert a["loss"] == b["loss"] and a["grad"] == b["grad"]
        else:
            assert np.array_equal(a["mu"], b["mu"])


def test_server_matches_direct_calls(env):
    torch, api, server = env
    kind, p, _ = _requests()[0]
    res, _ = _run(server, [(kind, p, None)], 2)
    opts = api.solve_opts(nprobe=6, nlanczos=15, cg_rtol=1e-6, seed=9, cg_maxit=400)
    loss, grad, _ = api.gp_loss_and_grad(torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda(),
                                         p.kind, p.theta, opts)
    assert res[0]["loss"] == loss and res[0]["grad"] == grad


def test_prediction_matches_oracle(env):
    torch, api, server = env
    p = inputs.uniform_problem(1200, 3, O.GAUSSIAN, (0.1, 1.0, 0.3), seed=21)
    Xs = inputs.points(500, 3, seed=22)
    res, _ = _run(server, [(1, p, Xs)], 1)
    assert res[0]["status"] == 0
    alpha = O.exact_nll(p.X, p.y, p.kind, p.theta)["alpha"]
    ref = O.predict_mean(p.X, Xs, alpha, p.kind, p.theta)
    # CG to 1e-6 on a system with kappa ~ 6e3 moves mu by ~kappa * 1e-6 relative at most.
    assert np.linalg.norm(res[0]["mu"] - ref) / np.linalg.norm(ref) <= 1e-3


def test_admission_respects_budget_and_refuses_oversize(env):
    torch, api, server = env
    reqs = _requests()
    with server.Server(1 << 30, 8) as srv:
        sizes = []
        for kind, p, Xs in reqs:
            r, keep = server.Server.request(kind, p.X, p.y, p.kind, p.theta, nprobe=6, Xstar=Xs,
                                            cg_maxit=400, nlanczos=15, cg_rtol=1e-6)
            sizes.append(srv.footprint(r))
    budget = 2 * max(sizes) + (1 << 20)
    res, stats = _run(server, reqs, 8, budget=budget)
    assert stats["peak_bytes"] <= stats["budget_bytes"]
    assert all(r["status"] in (0, 4) for r in res)
    from paper_2503_02259_gb300._binding import GPError
    big = inputs.uniform_problem(200000, 8, O.GAUSSIAN, (0.1, 1.0, 0.3), seed=1)
    with server.Server(64 << 20, 1) as srv:
        r, keep = server.Server.request(0, big.X, big.y, big.kind, big.theta, nprobe=16)
        with pytest.raises(GPError) as ei:
            srv.submit(r, keep)
        assert ei.value.status == 3   # GP_ERR_OOM
        assert srv.stats()["refused"] == 1


def test_least_work_first_admission(env):
    # One slot: A runs while B (larger) and C (smaller) queue; when A finishes,
    # the request with less work (C) starts before B.
    torch, api, server = env
    sizes = {"A": 20000, "B": 8000, "C": 1000}
    with server.Server(8 << 30, 1) as srv:
        tickets = {}
        for name in ("A", "B", "C"):
            p = inputs.uniform_problem(sizes[name], 3, O.GAUSSIAN, (0.1, 1.0, 0.3), seed=3)
            r, keep = server.Server.request(0, p.X, p.y, p.kind, p.theta, nprobe=4, cg_maxit=30,
                                            nlanczos=10, cg_rtol=1e-12)
            tickets[name] = srv.submit(r, keep)
        srv.drain(300)
        res = {k: srv.poll(t) for k, t in tickets.items()}
    assert all(r["status"] in (0, 4) for r in res.values())
    assert res["A"]["t_start"] <= res["C"]["t_start"] <= res["B"]["t_start"]


def _converged_requests():
    """n <= 4000, mixed d, kernels and kinds; Theta chosen so that kappa stays
    at a few 1e3 for the losses (measured 1e3 to 4e3) and near 30 for the
    predictions."""
    out = []
    specs = [  # (n, d, kernel, theta, kind)
        (1500, 2, O.GAUSSIAN, (0.1, 1.0, 0.2), 0),
        (3000, 3, O.MATERN32, (0.2, 1.2, 0.15), 0),
        (2200, 8, O.GAUSSIAN, (0.3, 0.8, 0.9), 0),
        (4000, 3, O.GAUSSIAN, (0.15, 1.0, 0.25), 0),
        (2500, 3, O.MATERN32, (1.0, 1.0, 0.08), 1),
        (1800, 2, O.GAUSSIAN, (1.0, 1.0, 0.05), 1),
    ]
    for i, (n, d, kern, theta, kind) in enumerate(specs):
        prob = inputs.uniform_problem(n, d, kern, theta, seed=40 + i)
        Xs = inputs.points(400, d, seed=60 + i) if kind == 1 else None
        out.append((kind, prob, Xs))
    return out


@pytest.mark.parametrize("prec,slq", [(0, 0), (4, 3)])
def test_served_results_match_oracle_when_converged(env, prec, slq):
    torch, api, server = env
    reqs = _converged_requests()
    nprobe, k, seed = 8, 25, 5
    with server.Server(8 << 30, 4) as srv:
        tickets = []
        for kind, p, Xs in reqs:
            r, keep = server.Server.request(kind, p.X, p.y, p.kind, p.theta, nprobe=nprobe, Xstar=Xs,
                                            cg_maxit=3000, nlanczos=k, cg_rtol=1e-7, seed=seed,
                                            prec=prec, slq_prec=slq)
            tickets.append(srv.submit(r, keep))
        srv.drain(300)
        res = [srv.poll(t) for t in tickets]
    for (kind, p, Xs), r in zip(reqs, res):
        assert r["status"] == 0, r
        if kind == 0:
            est = O.est_nll(p.X, p.y, p.kind, p.theta, O.rademacher_probes(p.n, nprobe, seed), k)
            assert abs(r["loss"] - est["loss"]) <= 1e-4 * abs(est["loss"])
            g = np.asarray(est["grad"])
            floor = 1e-3 * np.linalg.norm(g)
            for t in range(3):
                assert abs(r["grad"][t] - g[t]) <= 1e-4 * max(abs(g[t]), floor), (r["grad"], g)
        else:
            alpha = O.exact_nll(p.X, p.y, p.kind, p.theta)["alpha"]
            ref = O.predict_mean(p.X, Xs, alpha, p.kind, p.theta)
            assert np.linalg.norm(r["mu"] - ref) / np.linalg.norm(ref) <= 1e-4


def test_batched_server_gives_the_unbatched_results(env):
    # Loss + gradient requests with 16 probes (1 + p = 17 columns, a grouped
    # width) run as batches of up to 8 in one grouped launch per solver step;
    # every result equals the one-request-at-a-time server's bit for bit.
    torch, api, server = env
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(12):
        n = int(rng.integers(500, 2500))
        d = [2, 3][i % 2]
        prob = inputs.uniform_problem(n, d, O.GAUSSIAN, (0.1, 1.0, 0.25), seed=200 + i)
        reqs.append((0, prob, None))

    def run(max_batch, slots):
        with server.Server(8 << 30, slots, max_batch=max_batch) as srv:
            tickets = []
            for kind, p, Xs in reqs:
                r, keep = server.Server.request(kind, p.X, p.y, p.kind, p.theta, nprobe=16,
                                                cg_maxit=300, nlanczos=15, cg_rtol=1e-7, seed=4)
                tickets.append(srv.submit(r, keep))
            srv.drain(300)
            return [srv.poll(t) for t in tickets], srv.stats()

    plain, _ = run(1, 1)
    batched, stats = run(8, 1)
    assert stats["batches"] >= 1 and stats["largest_batch"] >= 2
    for a, b in zip(plain, batched):
        assert a["status"] == b["status"] == 0
        assert a["loss"] == b["loss"] and a["grad"] == b["grad"]
