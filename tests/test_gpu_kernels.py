"""GPU parity of the on-the-fly products against the FP64 oracle, called
through the C ABI.  Tolerance (FP32 path): max over columns of the norm-wise
relative error ||Y_gpu - Y_oracle||_2 / ||Y_oracle||_2 <= 1e-5, on all rows or
on the same sampled rows on both sides."""
import numpy as np
import pytest

import oracle as O
from paper_2503_02259_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def api():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import api as A
    return A


def colwise_relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.ndim == 1:
        got, ref = got[:, None], ref[:, None]
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1), num)))


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    # (n, d, w, kind)
    (1, 3, 1, O.GAUSSIAN),
    (2, 1, 4, O.MATERN32),
    (127, 2, 11, O.GAUSSIAN),
    (128, 3, 17, O.MATERN32),
    (129, 5, 32, O.GAUSSIAN),
    (300, 8, 33, O.MATERN32),
    (513, 3, 37, O.GAUSSIAN),      # one 40-column group (TW = 40)
    (640, 8, 40, O.MATERN32),
    (777, 16, 64, O.GAUSSIAN),
    (2000, 3, 11, O.GAUSSIAN),
    (2000, 3, 32, O.MATERN32),
    (1500, 4, 100, O.MATERN32),
    (1031, 2, 128, O.GAUSSIAN),
]


@pytest.mark.parametrize("n,d,w,kind", CASES)
def test_grad_matmul_matches_oracle(api, n, d, w, kind):
    theta = (0.05, 1.5, 0.2) if kind == O.MATERN32 else (0.1, 1.0, 0.3)
    X = inputs.points(n, d, seed=n + d)
    V = inputs.gaussian_block(n, w, seed=w)
    Y, dYf, dYl = api.gp_kernel_grad_matmul(_dev(X), _dev(V), kind, theta)
    rY, rF, rL = O.kmv_rows(X, V, kind, theta)
    assert colwise_relerr(Y.cpu().numpy(), rY) <= TOL_FP32
    assert colwise_relerr(dYf.cpu().numpy(), rF) <= TOL_FP32
    if n > 1:
        assert colwise_relerr(dYl.cpu().numpy(), rL) <= TOL_FP32
    else:
        assert np.all(dYl.cpu().numpy() == 0.0)


@pytest.mark.parametrize("n,d,w,kind", CASES[::2])
def test_matmul_matches_oracle(api, n, d, w, kind):
    theta = (0.2, 0.7, 0.45)
    X = inputs.points(n, d, seed=3 * n + d)
    V = inputs.gaussian_block(n, w, seed=5 + w)
    Y = api.gp_kernel_matmul(_dev(X), _dev(V), kind, theta)
    rY, _, _ = O.kmv_rows(X, V, kind, theta)
    assert colwise_relerr(Y.cpu().numpy(), rY) <= TOL_FP32


def test_matmul_equals_grad_matmul_first_output(api):
    X = inputs.points(1000, 3, seed=1)
    V = inputs.gaussian_block(1000, 20, seed=2)
    th = (0.05, 1.5, 0.2)
    Y1 = api.gp_kernel_matmul(_dev(X), _dev(V), O.MATERN32, th).cpu().numpy()
    Y2 = api.gp_kernel_grad_matmul(_dev(X), _dev(V), O.MATERN32, th)[0].cpu().numpy()
    assert colwise_relerr(Y1, Y2) <= 1e-6


def test_products_are_deterministic(api):
    X = _dev(inputs.points(3000, 3, seed=4))
    V = _dev(inputs.gaussian_block(3000, 32, seed=4))
    a = [t.cpu().numpy() for t in api.gp_kernel_grad_matmul(X, V, O.MATERN32, (0.05, 1.5, 0.2))]
    b = [t.cpu().numpy() for t in api.gp_kernel_grad_matmul(X, V, O.MATERN32, (0.05, 1.5, 0.2))]
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_identical_points_closed_form(api, kind):
    # All points equal: Kh V = f^2 1 (1^T V) + s V, dKh/dl V = 0.
    n, w, s, f = 517, 9, 0.2, 1.7
    X = np.full((n, 3), 0.37, dtype=np.float32)
    V = inputs.gaussian_block(n, w, seed=8)
    Y, dYf, dYl = api.gp_kernel_grad_matmul(_dev(X), _dev(V), kind, (s, f, 0.3))
    ref = f * f * V.astype(np.float64).sum(axis=0)[None, :] + s * V
    assert colwise_relerr(Y.cpu().numpy(), ref) <= TOL_FP32
    assert np.abs(dYl.cpu().numpy()).max() == 0.0


@pytest.mark.parametrize("kind", [O.GAUSSIAN, O.MATERN32])
def test_far_points_closed_form(api, kind):
    n, w, s, f, l = 300, 5, 0.2, 1.7, 0.01
    X = np.zeros((n, 2), dtype=np.float32)
    X[:, 0] = 50 * l * np.arange(n)
    V = inputs.gaussian_block(n, w, seed=9)
    Y = api.gp_kernel_matmul(_dev(X), _dev(V), kind, (s, f, l)).cpu().numpy()
    assert colwise_relerr(Y, (f * f + s) * V.astype(np.float64)) <= TOL_FP32


def test_fused_matvec_config_sampled_rows(api):
    # n = 1e5, d = 3, Matern-3/2 (f = 1.5, l = 0.2, s = 0.05), V = [y | 31 Rademacher].
    prob = inputs.matvec_problem(seed=0)
    V = inputs.multivector(prob.y, 32, seed=0)
    Y, dYf, dYl = api.gp_kernel_grad_matmul(_dev(prob.X), _dev(V), prob.kind, prob.theta)
    rows = np.sort(np.random.default_rng(0).choice(prob.n, 1000, replace=False))
    rY, rF, rL = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows, block=100)
    assert colwise_relerr(Y.cpu().numpy()[rows], rY) <= TOL_FP32
    assert colwise_relerr(dYf.cpu().numpy()[rows], rF) <= TOL_FP32
    assert colwise_relerr(dYl.cpu().numpy()[rows], rL) <= TOL_FP32


def test_probe_generator_bit_exact(api):
    for n, p, seed in [(1, 1, 0), (1000, 7, 12345), (4099, 33, 2**63 + 17)]:
        Z = api.gp_generate_probes(n, p, seed).cpu().numpy()
        assert np.array_equal(Z, O.rademacher_probes(n, p, seed))


@pytest.mark.parametrize("m,n,d,kind", [(1, 50, 3, O.GAUSSIAN), (1000, 2000, 3, O.MATERN32),
                                        (129, 4097, 8, O.GAUSSIAN)])
def test_predict_mean_matches_oracle(api, m, n, d, kind):
    theta = (0.1, 1.3, 0.4)
    X = inputs.points(n, d, seed=m)
    Xs = inputs.points(m, d, seed=m + 1)
    alpha = inputs.gaussian_block(n, 1, seed=m)[:, 0]
    mu = api.gp_predict_mean(_dev(X), _dev(alpha), _dev(Xs), kind, theta).cpu().numpy()
    ref = O.predict_mean(X, Xs, alpha, kind, theta)
    assert colwise_relerr(mu, ref) <= TOL_FP32


def test_bad_arguments_raise(api):
    import torch
    from paper_2503_02259_gb300._binding import GPError
    X = torch.zeros((10, 3), device="cuda")
    V = torch.zeros((10, 129), device="cuda")
    with pytest.raises((GPError, ValueError)):
        api.gp_kernel_matmul(X, V, 0, (0.1, 1.0, 0.3))
    with pytest.raises((GPError, ValueError)):
        api.gp_kernel_matmul(X, V[:, :4], 0, (0.1, 1.0, -0.3))


def test_pipe_rate_microbenchmarks_are_plausible(api):
    # The FP32 pipe of a GB300 (152 SMs x 128 lanes x 2 flops x up to 2.07 GHz
    # = 80.5 TFLOP/s) and its MUFU unit: the measured rates must be positive,
    # below the unit-count bound, and within a factor 4 of it (clocks vary).
    from paper_2503_02259_gb300 import _binding as B
    import torch
    f, m = B.c_double(), B.c_double()
    B.check(B.lib().gp_measure_pipe_rates(B.ctypes.byref(f), B.ctypes.byref(m),
                                          torch.cuda.current_stream().cuda_stream),
            "gp_measure_pipe_rates")
    props = torch.cuda.get_device_properties(0)
    bound = props.multi_processor_count * 128 * 2 * 2.1e9 / 1e12
    assert bound / 4 < f.value <= bound * 1.02
    assert m.value > 100.0
