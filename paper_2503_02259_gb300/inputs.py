"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module draws points, targets and right-hand sides only; it holds none
of the method's arithmetic (no kernel, solver or estimator).  Every array is
produced in float64 by ``numpy.random.default_rng(seed)`` and cast to
float32, the precision the library consumes.

The paper measures on UCI Bike, UCI 3D Road Network and three synthetic
test functions from the Virtual Library of Simulation Experiments
(§Numerical Experiments); none is available here, so these seeded recipes
stand in for them at the paper's scales and kernels (RBF, Matern-3/2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAUSSIAN = 0
MATERN32 = 1


@dataclasses.dataclass
class Problem:
    X: np.ndarray          # (n, d) float32, row-major
    y: np.ndarray          # (n,) float32
    kind: int              # GAUSSIAN or MATERN32
    theta: tuple           # (s, f, l)

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def _target_sincos(X: np.ndarray, rng) -> np.ndarray:
    """y = sin(2 pi x1) cos(2 pi x2) + x3 + 0.1 N(0,1) on the first min(d,3) coordinates."""
    d = X.shape[1]
    t = np.sin(2 * math.pi * X[:, 0])
    if d >= 2:
        t = t * np.cos(2 * math.pi * X[:, 1])
    if d >= 3:
        t = t + X[:, 2]
    return t + 0.1 * rng.standard_normal(X.shape[0])


def uniform_problem(n: int, d: int, kind: int, theta, seed: int = 0) -> Problem:
    """X ~ U[0,1]^d, y from the sin/cos target above."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    y = _target_sincos(X, rng)
    return Problem(X.astype(np.float32), y.astype(np.float32), kind, tuple(theta))


def small_problem(seed: int = 0, n: int = 2000) -> Problem:
    """Plain method, small: n=2000, d=3 uniform, Gaussian f=1, l=0.3, s=0.1."""
    return uniform_problem(n, 3, GAUSSIAN, (0.1, 1.0, 0.3), seed)


def matvec_problem(seed: int = 0, n: int = 100_000) -> Problem:
    """Fused matvec throughput: n=1e5, d=3 uniform, Matern-3/2 f=1.5, l=0.2, s=0.05."""
    return uniform_problem(n, 3, MATERN32, (0.05, 1.5, 0.2), seed)


def precision_problem(seed: int = 0, n: int = 1_000_000) -> Problem:
    """Precision: n=1e6, d=2 uniform, Gaussian f=1, l=0.05, s=0.01 (ill-conditioned)."""
    return uniform_problem(n, 2, GAUSSIAN, (0.01, 1.0, 0.05), seed)


def diff_problem(seed: int = 0, n: int = 200_000) -> Problem:
    """Differentiation: n=2e5, d=8, x ~ 0.5 N(0,I); y = sum_k sin(x_k)/8 + 0.05 N(0,1);
    Gaussian s=0.1, f=1, l=1.2."""
    rng = np.random.default_rng(seed)
    X = 0.5 * rng.standard_normal((n, 8))
    y = np.sin(X).sum(axis=1) / 8.0 + 0.05 * rng.standard_normal(n)
    return Problem(X.astype(np.float32), y.astype(np.float32), GAUSSIAN, (0.1, 1.0, 1.2))


def multivector(y: np.ndarray, w: int, seed: int = 0) -> np.ndarray:
    """V = [y | w-1 Rademacher columns] as float32 (n, w), row-major."""
    rng = np.random.default_rng(seed + 7919)
    n = y.shape[0]
    V = np.empty((n, w), dtype=np.float32)
    V[:, 0] = y
    if w > 1:
        V[:, 1:] = rng.integers(0, 2, size=(n, w - 1)) * 2.0 - 1.0
    return V


def gaussian_block(n: int, w: int, seed: int = 0) -> np.ndarray:
    """A dense N(0,1) float32 block (n, w) for generic matvec tests."""
    return np.random.default_rng(seed + 104729).standard_normal((n, w)).astype(np.float32)


def points(n: int, d: int, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """n points uniform on [0, scale]^d, float32."""
    return (scale * np.random.default_rng(seed + 31).random((n, d))).astype(np.float32)


@dataclasses.dataclass
class Request:
    t_arrive: float        # seconds after the stream start
    kind: int              # 0 = loss+grad, 1 = predict
    problem: Problem
    Xstar: np.ndarray | None
    nprobe: int


def serving_stream(seed: int = 0, count: int = 512, rate: float = 50.0,
                   n_lo: int = 1_000, n_hi: int = 300_000, m: int = 10_000,
                   nprobe: int = 16) -> list[Request]:
    """Poisson stream of mixed requests: n log-uniform in [n_lo, n_hi], d in {2,3,8},
    X ~ U[0,1]^d, Gaussian or Matern-3/2, l ~ logU[0.05,1], s ~ logU[1e-3,0.3],
    f ~ logU[0.5,2]; 70% loss+grad, 30% prediction at m test points."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.choice([2, 3, 8]))
        kind = int(rng.integers(0, 2))
        l = math.exp(rng.uniform(math.log(0.05), math.log(1.0)))
        s = math.exp(rng.uniform(math.log(1e-3), math.log(0.3)))
        f = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
        rkind = 0 if rng.random() < 0.7 else 1
        X = rng.random((n, d))
        y = _target_sincos(X, rng)
        prob = Problem(X.astype(np.float32), y.astype(np.float32), kind, (s, f, l))
        Xs = rng.random((m, d)).astype(np.float32) if rkind == 1 else None
        out.append(Request(t, rkind, prob, Xs, nprobe))
    return out
