"""GPU parity of the tcgen05 tensor-core product against the FP64 oracle.

Tolerances (norm-wise per column, as for the FP32 tests):
  * TF32 operands, FP32 accumulation: <= 3e-3, the tile bound of the
    mixed-precision path before refinement;
  * split TF32 (hi*hi + hi*lo + lo*hi): <= 1e-5, the FP32 bound;
  * split BF16: <= 3e-5 (a 16-bit hi + lo pair leaves 2^-17 per entry); this
    is the BF16-operand path that meets the tile bound;
  * plain BF16 (kernel tile rounded once to BF16, V as hi + lo): NOT within
    the 3e-3 tile bound and not claimed for it.  An entry rounded to 8
    significant bits carries about 1.7e-3 rms relative error, and products
    with a probe column whose result cancels reach 2e-3 to 6e-3 (a CPU
    simulation of the rounding on these cases gives up to 3.5e-3 for K-hat V
    and 5.7e-3 for dK-hat/dl V); it is held here to 1e-2, as the fast
    low-accuracy mode that it is.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_02259_gb300 import inputs

pytestmark = pytest.mark.gpu

TILE_BOUND = 3e-3
TOL = {1: TILE_BOUND, 2: 1e-2, 3: 1e-5, 4: 3e-5}   # TF32, BF16 (outside the tile bound), TF32X3, BF16X3
MODES = [1, 2, 3, 4]


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


def colwise_relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.ndim == 1:
        got, ref = got[:, None], ref[:, None]
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


@pytest.mark.parametrize("prec", MODES)
def test_tc_smallest_tile(api, prec):
    # One 128-row tile, four 32-point column tiles, N = 16.
    n, w = 128, 16
    X = inputs.points(n, 3, seed=1)
    V = inputs.gaussian_block(n, w, seed=1)
    theta = (0.1, 1.0, 0.3)
    Y = api.gp_kernel_matmul(_dev(X), _dev(V), O.GAUSSIAN, theta, prec=prec).cpu().numpy()
    rY, _, _ = O.kmv_rows(X, V, O.GAUSSIAN, theta)
    assert colwise_relerr(Y, rY) <= TOL[prec]


CASES = [
    (1, 2, 1, O.GAUSSIAN),
    (127, 3, 17, O.MATERN32),
    (300, 8, 32, O.GAUSSIAN),
    (2000, 3, 11, O.GAUSSIAN),
    (2000, 2, 64, O.MATERN32),
    (1537, 16, 33, O.MATERN32),
    (1031, 4, 128, O.GAUSSIAN),
]


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("n,d,w,kind", CASES)
def test_tc_grad_matmul_matches_oracle(api, prec, n, d, w, kind):
    theta = (0.05, 1.5, 0.2) if kind == O.MATERN32 else (0.1, 1.0, 0.3)
    X = inputs.points(n, d, seed=n + d)
    V = inputs.gaussian_block(n, w, seed=w)
    import torch
    Xd, Vd = _dev(X), _dev(V)
    prob, _ = api.problem(Xd, kind, theta)
    Y = torch.empty_like(Vd)
    dYf = torch.empty_like(Vd)
    dYl = torch.empty_like(Vd)
    from paper_2503_02259_gb300 import _binding as B
    ws = api.workspace(B.OP_GRAD_MATMUL, prob, w, api.solve_opts(prec=prec), Xd.device)
    B.check(B.lib().gp_kernel_grad_matmul(B.ctypes.byref(prob), api._ptr(Vd), w, api._ptr(Y),
                                          api._ptr(dYf), api._ptr(dYl), prec, api._ptr(ws),
                                          ws.numel(), api._stream(Xd.device)), "grad_matmul")
    rY, rF, rL = O.kmv_rows(X, V, kind, theta)
    assert colwise_relerr(Y.cpu().numpy(), rY) <= TOL[prec]
    assert colwise_relerr(dYf.cpu().numpy(), rF) <= TOL[prec]
    if n > 1:
        assert colwise_relerr(dYl.cpu().numpy(), rL) <= TOL[prec]


@pytest.mark.parametrize("prec", MODES)
def test_tc_precision_config_sampled_rows(api, prec):
    # n = 1e6, d = 2 uniform, Gaussian f = 1, l = 0.05, s = 0.01, V width 64.
    prob = inputs.precision_problem(seed=0)
    V = inputs.multivector(prob.y, 64, seed=0)
    Y = api.gp_kernel_matmul(_dev(prob.X), _dev(V), prob.kind, prob.theta, prec=prec).cpu().numpy()
    rows = np.sort(np.random.default_rng(3).choice(prob.n, 1000, replace=False))
    rY, _, _ = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows, block=20)
    assert colwise_relerr(Y[rows], rY) <= TOL[prec]


@pytest.mark.parametrize("prec", [3, 4])
def test_tc_split_matches_oracle_at_fused_matvec_size(api, prec):
    # n = 1e5, d = 3 uniform, Matern-3/2: long accumulation chains per row.
    prob = inputs.matvec_problem(seed=0)
    V = inputs.multivector(prob.y, 32, seed=0)
    Y = api.gp_kernel_matmul(_dev(prob.X), _dev(V), prob.kind, prob.theta, prec=prec).cpu().numpy()
    rows = np.sort(np.random.default_rng(5).choice(prob.n, 500, replace=False))
    rY, _, _ = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows, block=100)
    assert colwise_relerr(Y[rows], rY) <= TOL[prec]


# Split BF16 on point clouds unlike the uniform cubes above, at d in 5..16
# without the derivative: compact Gaussian clouds, a spread cube at a short
# length-scale, and clouds with far outliers.  On the clustered clouds K-hat is
# close to a constant matrix and K-hat V cancels (|K-hat V| at most 0.09 of
# K-hat |V| here), so the rounding of the entries, relative to the entries, is
# bounded against K-hat |V|: measured up to 5.2e-5 of |K-hat V|, at most 3.6e-6
# of K-hat |V|.  The product without the derivative and the K-hat V of the
# derivative product share the evaluation and the split arithmetic: they agree
# to 1e-5.
def _cloud(kind, n, d, seed):
    rng = np.random.default_rng(seed)
    if kind == "compact":
        return (0.5 * rng.standard_normal((n, d))).astype(np.float32)
    if kind == "spread":
        return rng.random((n, d)).astype(np.float32)
    X = 0.3 * rng.standard_normal((n, d))
    far = rng.random(n) < 0.03
    X[far] += 2.5
    return X.astype(np.float32)


@pytest.mark.parametrize("n,d,w,kind,cloud,l", [
    (1000, 8, 33, O.GAUSSIAN, "compact", 1.2),
    (1537, 16, 48, O.MATERN32, "compact", 3.0),
    (129, 8, 16, O.GAUSSIAN, "compact", 1.2),
    (300, 8, 16, O.GAUSSIAN, "spread", 0.3),
    (2000, 8, 128, O.MATERN32, "outliers", 1.5),
    (777, 5, 20, O.GAUSSIAN, "outliers", 1.0),
])
def test_tc_split_bf16_on_clustered_clouds(api, n, d, w, kind, cloud, l):
    X = _cloud(cloud, n, d, seed=n + d)
    V = inputs.gaussian_block(n, w, seed=w + 1)
    theta = (0.1, 1.0, l)
    Y = api.gp_kernel_matmul(_dev(X), _dev(V), kind, theta, prec=4).cpu().numpy()
    rY, _, _ = O.kmv_rows(X.astype(np.float64), V, kind, theta)
    rA, _, _ = O.kmv_rows(X.astype(np.float64), np.abs(V), kind, theta)   # K-hat |V|
    err = np.linalg.norm(Y - rY, axis=0) / np.linalg.norm(rA, axis=0)
    assert float(err.max()) <= TOL[4]
    # The derivative product's K-hat V.
    import torch
    Xd, Vd = _dev(X), _dev(V)
    prob, _ = api.problem(Xd, kind, theta)
    Y2 = torch.empty_like(Vd)
    dYf = torch.empty_like(Vd)
    from paper_2503_02259_gb300 import _binding as B
    ws = api.workspace(B.OP_GRAD_MATMUL, prob, w, api.solve_opts(prec=4), Xd.device)
    B.check(B.lib().gp_kernel_grad_matmul(B.ctypes.byref(prob), api._ptr(Vd), w, api._ptr(Y2),
                                          api._ptr(dYf), None, 4, api._ptr(ws), ws.numel(),
                                          api._stream(Xd.device)), "grad_matmul")
    assert colwise_relerr(Y, Y2.cpu().numpy()) <= 1e-5
