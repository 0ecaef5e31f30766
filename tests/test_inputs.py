"""The seeded input recipes match the workloads they stand in for: sizes,
dimensions, kernels, hyper-parameters and value distributions."""
import math

import numpy as np

from paper_2503_02259_gb300 import inputs


def test_fixed_problems_have_the_configured_shapes_and_parameters():
    p = inputs.small_problem(seed=0)
    assert (p.n, p.d, p.kind, p.theta) == (2000, 3, inputs.GAUSSIAN, (0.1, 1.0, 0.3))
    assert p.X.dtype == np.float32 and 0.0 <= p.X.min() and p.X.max() <= 1.0
    p = inputs.matvec_problem(seed=0, n=5000)
    assert (p.d, p.kind, p.theta) == (3, inputs.MATERN32, (0.05, 1.5, 0.2))
    p = inputs.precision_problem(seed=0, n=5000)
    assert (p.d, p.kind, p.theta) == (2, inputs.GAUSSIAN, (0.01, 1.0, 0.05))
    p = inputs.diff_problem(seed=0, n=20000)
    assert (p.d, p.kind, p.theta) == (8, inputs.GAUSSIAN, (0.1, 1.0, 1.2))
    # x ~ 0.5 N(0, I): per-coordinate standard deviation 0.5.
    assert abs(float(p.X.std()) - 0.5) < 0.01 and abs(float(p.X.mean())) < 0.01
    # The n = 4000 subsample is the first 4000 rows of the same seeded draw.
    sub = inputs.diff_problem(seed=0, n=4000)
    assert sub.n == 4000 and np.isfinite(sub.y).all()


def test_target_follows_the_sincos_recipe():
    p = inputs.small_problem(seed=1)
    X = p.X.astype(np.float64)
    clean = np.sin(2 * math.pi * X[:, 0]) * np.cos(2 * math.pi * X[:, 1]) + X[:, 2]
    noise = p.y.astype(np.float64) - clean
    assert abs(noise.std() - 0.1) < 0.01 and abs(noise.mean()) < 0.01


def test_multivector_is_y_then_rademacher():
    y = np.arange(100, dtype=np.float32)
    V = inputs.multivector(y, 32, seed=0)
    assert V.shape == (100, 32) and np.array_equal(V[:, 0], y)
    assert set(np.unique(V[:, 1:])) == {-1.0, 1.0}


def test_serving_stream_follows_the_recipe():
    reqs = inputs.serving_stream(seed=0, count=48, n_hi=20_000)
    t = np.array([r.t_arrive for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 0.5 / 50 < np.diff(t).mean() < 2.0 / 50          # Poisson at 50 per second
    for r in reqs:
        p = r.problem
        assert 1000 <= p.n <= 20000 and p.d in (2, 3, 8)
        assert p.kind in (inputs.GAUSSIAN, inputs.MATERN32)
        s, f, l = p.theta
        assert 1e-3 <= s <= 0.3 and 0.5 <= f <= 2.0 and 0.05 <= l <= 1.0
        assert r.nprobe == 16
        if r.kind == 1:
            assert r.Xstar.shape == (10_000, p.d)
        else:
            assert r.Xstar is None
    share = np.mean([r.kind == 0 for r in reqs])
    assert 0.45 < share < 0.95                                # 70 % loss+grad
