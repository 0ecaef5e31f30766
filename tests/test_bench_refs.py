"""The FP64 reference values bench.py compares against (tests/golden/bench_refs.npz,
written by tests/golden/make_bench_refs.py) are the oracle's: recompute a few of
them here and compare."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2503_02259_gb300 import inputs

REFS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bench_refs.npz")


def test_matvec_rows_are_the_oracles():
    refs = np.load(REFS)
    prob = inputs.matvec_problem(seed=0)
    V = inputs.multivector(prob.y, 32, seed=0)
    rows = np.sort(np.random.default_rng(11).choice(prob.n, 100, replace=False))
    assert np.array_equal(rows, refs["matvec_rows"])
    Y, _, Lr = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows[:3], block=3)
    np.testing.assert_allclose(Y, refs["matvec_Y"][:3], rtol=1e-12, atol=0)
    np.testing.assert_allclose(Lr, refs["matvec_L"][:3], rtol=1e-12, atol=0)


def test_precision_rows_are_the_oracles():
    refs = np.load(REFS)
    prob = inputs.precision_problem(seed=0)
    V = inputs.multivector(prob.y, 64, seed=0)
    rows = np.sort(np.random.default_rng(3).choice(prob.n, 200, replace=False))
    assert np.array_equal(rows, refs["precision_rows"])
    Y, _, _ = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows[-2:], block=2)
    np.testing.assert_allclose(Y, refs["precision_Y"][-2:], rtol=1e-12, atol=0)


def test_differentiation_subsample_estimate_is_the_oracles():
    refs = np.load(REFS)
    sub = inputs.diff_problem(seed=0, n=4000)
    est = O.est_nll(sub.X, sub.y, sub.kind, sub.theta, O.rademacher_probes(sub.n, 32, 77), 40)
    assert abs(est["loss"] - float(refs["diff_loss"])) <= 1e-9 * abs(est["loss"])
    np.testing.assert_allclose(est["grad"], refs["diff_grad"], rtol=1e-9, atol=0)


def test_serving_references_are_the_oracles():
    refs = np.load(REFS)
    reqs = inputs.serving_stream(seed=0, count=512)
    idx = refs["serving_idx"]
    assert len(idx) == 24 and all(reqs[int(i)].problem.n <= 3000 for i in idx)
    # The first loss+grad request and the first prediction of the selection.
    k_loss = next(k for k, i in enumerate(idx) if reqs[int(i)].kind == 0)
    k_pred = next(k for k, i in enumerate(idx) if reqs[int(i)].kind == 1)
    rq = reqs[int(idx[k_loss])]
    p = rq.problem
    est = O.est_nll(p.X, p.y, p.kind, p.theta, O.rademacher_probes(p.n, rq.nprobe, 0), 20)
    assert abs(est["loss"] - float(refs["serving_loss"][k_loss])) <= 1e-9 * abs(est["loss"])
    np.testing.assert_allclose(est["grad"], refs["serving_grad"][k_loss], rtol=1e-9, atol=0)
    rq = reqs[int(idx[k_pred])]
    p = rq.problem
    alpha = O.exact_nll(p.X, p.y, p.kind, p.theta)["alpha"]
    mu = O.predict_mean(p.X, rq.Xstar[:200], alpha, p.kind, p.theta)
    np.testing.assert_allclose(mu, refs["serving_mu"][k_pred], rtol=1e-9, atol=1e-12)
    assert np.isnan(refs["serving_loss"][k_pred]) and np.isnan(refs["serving_mu"][k_loss]).all()


def test_serving_condition_numbers_are_the_oracles():
    refs = np.load(REFS)
    reqs = inputs.serving_stream(seed=0, count=512)
    k = 3
    p = reqs[int(refs["serving_idx"][k])].problem
    ev = np.linalg.eigvalsh(O.khat_dense(p.X, p.kind, p.theta))
    assert ev[-1] / ev[0] == pytest.approx(float(refs["serving_kappa"][k]), rel=1e-9)


def test_precision_subsample_exact_loss_is_the_oracles():
    refs = np.load(REFS)
    sub = inputs.precision_problem(seed=0, n=4000)
    ex = O.exact_nll(sub.X, sub.y, sub.kind, sub.theta)
    assert abs(ex["loss"] - float(refs["preck_loss"])) <= 1e-9 * abs(ex["loss"])
    np.testing.assert_allclose(ex["grad"], refs["preck_grad"], rtol=1e-9, atol=0)


def test_differentiation_subsample_exact_loss_is_the_oracles():
    refs = np.load(REFS)
    sub = inputs.diff_problem(seed=0, n=4000)
    ex = O.exact_nll(sub.X, sub.y, sub.kind, sub.theta)
    assert abs(ex["loss"] - float(refs["diffx_loss"])) <= 1e-9 * abs(ex["loss"])
    np.testing.assert_allclose(ex["grad"], refs["diffx_grad"], rtol=1e-9, atol=0)
