"""gp_kernel_matmul_noalloc: the product for callers that cannot allocate.

Some callers of this library cannot call cudaMalloc at the point where they
need the product: a plug-in running inside a host application (an inference
server, another framework's custom-op hook) whose host owns the device
allocator and forbids allocation in its execute callback, or a loop with a
fixed memory budget that must not allocate once it has started.  For them the
library keeps its scratch in one static device array.  These tests call that
entry point through the C ABI and compare it with gp_kernel_matmul, the
workspace entry point, and with the FP64 oracle, within the FP32 product
tolerance used by the other product tests (norm-wise 1e-5 per column), on
calls in a row with different shapes (a smaller problem, then one whose w
needs no padding, after a larger one), so that stale contents of the shared
array would show; and on a second stream, ordered after the first by a
synchronize, which reuses the device address looked up by the first call.

This file is collected last on purpose (its name sorts last), and it passes
both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import _binding as B
    from paper_2503_02259_gb300 import api, inputs
    return torch, B, api, inputs


def _relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


def _noalloc(env, X, V, kind, theta):
    torch, B, api, _ = env
    prob, X = api.problem(X, kind, theta)
    Y = torch.full_like(V, float("nan"))
    st = B.lib().gp_kernel_matmul_noalloc(ctypes.byref(prob), ctypes.c_void_p(V.data_ptr()),
                                          V.shape[1], ctypes.c_void_p(Y.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    B.check(st, "gp_kernel_matmul_noalloc")
    torch.cuda.synchronize()
    return Y


def test_noalloc_matches_workspace_entry_point_two_calls(env):
    torch, B, api, inputs = env
    cases = [
        (20000, 3, 32, 1, (0.05, 1.5, 0.2)),   # Matern-3/2, full-width columns
        (3001, 2, 11, 0, (0.1, 1.0, 0.3)),     # Gaussian, ragged n and padded w
    ]
    for n, d, w, kind, theta in cases:
        X = torch.from_numpy(inputs.points(n, d, seed=n)).cuda()
        V = torch.from_numpy(inputs.gaussian_block(n, w, seed=w)).cuda()
        ref = api.gp_kernel_matmul(X, V, kind, theta).cpu().numpy()
        got = _noalloc(env, X, V, kind, theta).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _relerr(got, ref) <= TOL_FP32


def test_noalloc_matches_oracle_after_larger_calls(env):
    import oracle as O
    torch, B, api, inputs = env
    # A large call leaves the shared array dirty beyond what the next ones use.
    Xb = torch.from_numpy(inputs.points(40000, 3, seed=1)).cuda()
    Vb = torch.from_numpy(inputs.gaussian_block(40000, 40, seed=2)).cuda()
    _noalloc(env, Xb, Vb, 1, (0.05, 1.5, 0.2))
    cases = [
        (2999, 3, 32, 1, (0.05, 1.5, 0.2)),    # w = w_pad: no padded columns to re-zero
        (1531, 2, 7, 0, (0.1, 1.0, 0.3)),      # ragged n, padded w
    ]
    for n, d, w, kind, theta in cases:
        Xh = inputs.points(n, d, seed=n + 1)
        Vh = inputs.gaussian_block(n, w, seed=w + 1)
        ref = O.kmv_rows(Xh, Vh, kind, theta)[0]
        got = _noalloc(env, torch.from_numpy(Xh).cuda(), torch.from_numpy(Vh).cuda(), kind,
                       theta).cpu().numpy()
        assert _relerr(got, ref) <= TOL_FP32


def test_noalloc_on_a_second_stream(env):
    import oracle as O
    torch, B, api, inputs = env
    n, d, w, kind, theta = 2500, 3, 16, 0, (0.1, 1.0, 0.3)
    Xh = inputs.points(n, d, seed=5)
    Vh = inputs.gaussian_block(n, w, seed=6)
    X = torch.from_numpy(Xh).cuda()
    V = torch.from_numpy(Vh).cuda()
    first = _noalloc(env, X, V, kind, theta)          # default stream, then synchronised
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        second = _noalloc(env, X, V, kind, theta)     # the same array on another stream
    torch.cuda.synchronize()
    assert torch.equal(first, second)
    assert _relerr(second.cpu().numpy(), O.kmv_rows(Xh, Vh, kind, theta)[0]) <= TOL_FP32


def test_noalloc_rejects_oversize_problem(env):
    torch, B, api, inputs = env
    X = torch.zeros((400000, 3), device="cuda")
    V = torch.zeros((400000, 32), device="cuda")
    prob, X = api.problem(X, 0, (0.1, 1.0, 0.3))
    st = B.lib().gp_kernel_matmul_noalloc(ctypes.byref(prob), ctypes.c_void_p(V.data_ptr()), 32,
                                          ctypes.c_void_p(V.data_ptr()), None)
    assert st == B.GP_ERR_ARG
    assert b"static scratch" in B.lib().gp_last_error()
