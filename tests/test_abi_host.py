"""CPU-only checks of the C ABI: the library builds, loads, exports every
function declared in include/gp.h, and rejects bad arguments without touching
a GPU.  Also the host build of the device's tridiagonal eigensolver against
LAPACK."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gp.h")


@pytest.fixture(scope="module")
def L():
    from paper_2503_02259_gb300 import build
    build.build()
    from paper_2503_02259_gb300 import _binding
    return _binding.lib()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for need in ["gp_kernel_matmul", "gp_kernel_grad_matmul", "gp_pcg_solve", "gp_slq_logdet",
                 "gp_loss_and_grad", "gp_predict_mean", "gp_workspace_bytes", "gp_last_error"]:
        assert need in names


def test_library_exports_every_declared_symbol(L):
    from paper_2503_02259_gb300 import _binding
    names = _declared_functions()
    for name in names:
        assert hasattr(L, name), name
        assert name in _binding.PROTOTYPES, name
    nm = subprocess.run(["nm", "-D", "--defined-only", _binding.LIB_PATH], capture_output=True,
                        text=True).stdout
    exported = set(re.findall(r"\bT (gp_[a-z_0-9]+)", nm))
    assert set(names) <= exported


def test_version_and_status_strings(L):
    assert b"sm_103a" in L.gp_version()
    assert L.gp_status_string(0) == b"GP_OK"
    assert L.gp_status_string(4) == b"GP_ERR_NOT_CONVERGED"


def test_argument_errors_need_no_gpu(L):
    from paper_2503_02259_gb300 import _binding as B
    prob = B.gp_problem(0, 10, 3, 0, B.gp_theta(0.1, 1.0, 0.3))
    st = L.gp_kernel_matmul(ctypes.byref(prob), None, 4, None, 0, None, 0, None)
    assert st == B.GP_ERR_ARG
    assert b"X is NULL" in L.gp_last_error()
    prob.X = 256
    prob.theta.l = -1.0
    assert L.gp_kernel_matmul(ctypes.byref(prob), None, 4, None, 0, None, 0, None) == B.GP_ERR_ARG
    assert b"theta" in L.gp_last_error()
    prob.theta.l = 0.3
    prob.d = 17
    assert L.gp_workspace_bytes(B.OP_MATMUL, ctypes.byref(prob), 4, None) == 0
    prob.d = 3
    assert L.gp_workspace_bytes(B.OP_MATMUL, ctypes.byref(prob), 129, None) == 0
    assert L.gp_workspace_bytes(B.OP_MATMUL, ctypes.byref(prob), 32, None) > 0
    opts = B.gp_solve_opts(nprobe=10, nlanczos=65)
    assert L.gp_workspace_bytes(B.OP_LOSS_GRAD, ctypes.byref(prob), 0, ctypes.byref(opts)) == 0
    opts.nlanczos = 30
    assert L.gp_workspace_bytes(B.OP_LOSS_GRAD, ctypes.byref(prob), 0, ctypes.byref(opts)) > 0
    # slq_prec: a precision or GP_PREC_SAME (-1); anything else is refused.
    for bad in (-2, 5, 99):
        opts.slq_prec = bad
        assert L.gp_workspace_bytes(B.OP_LOSS_GRAD, ctypes.byref(prob), 0, ctypes.byref(opts)) == 0
        assert b"slq_prec" in L.gp_last_error()
    opts.slq_prec = B.PREC_SAME
    assert L.gp_workspace_bytes(B.OP_LOSS_GRAD, ctypes.byref(prob), 0, ctypes.byref(opts)) > 0
    # A workspace that is too small is refused before any launch.
    prob.theta.l = 0.3
    st = L.gp_kernel_matmul(ctypes.byref(prob), 256, 4, 512, 0, 1024, 16, None)
    assert st == B.GP_ERR_OOM


def test_preconditioner_arguments_need_no_gpu(L):
    from paper_2503_02259_gb300 import _binding as B
    prob = B.gp_problem(256, 1000, 3, 0, B.gp_theta(0.1, 1.0, 0.3))
    opts = B.gp_solve_opts(nprobe=4, nlanczos=10, precond_rank=50)
    # SLQ alone and the split forward / backward calls do not take the preconditioner.
    assert L.gp_workspace_bytes(B.OP_SLQ, ctypes.byref(prob), 0, ctypes.byref(opts)) == 0
    assert b"Nystrom" in L.gp_last_error()
    st = L.gp_nll_forward(ctypes.byref(prob), 256, ctypes.byref(opts), 256, None, None, 256, 1 << 20,
                          None)
    assert st == B.GP_ERR_UNIMPLEMENTED
    # The loss takes it (isotropic only): its workspace grows by the factor, its
    # derivative, the Lanczos M-images and the work planes.
    plain = B.gp_solve_opts(nprobe=4, nlanczos=10)
    lb = L.gp_workspace_bytes(B.OP_LOSS_GRAD, ctypes.byref(prob), 0, ctypes.byref(plain))
    lp = L.gp_workspace_bytes(B.OP_LOSS_GRAD, ctypes.byref(prob), 0, ctypes.byref(opts))
    assert lb > 0 and lp - lb >= 2 * 4 * 1024 * 50 + 11 * 4 * 1024 * 8
    ls = (ctypes.c_double * 3)(0.3, 0.4, 0.5)
    prob.ls = ctypes.cast(ls, ctypes.c_void_p)
    st = L.gp_loss_and_grad(ctypes.byref(prob), 256, ctypes.byref(opts), None, None, None, 256, 1 << 20,
                            None)
    assert st == B.GP_ERR_UNIMPLEMENTED and b"isotropic" in L.gp_last_error()
    prob.ls = None
    # The solve's workspace holds at least the factor's FP32 columns.
    base = L.gp_workspace_bytes(B.OP_PCG, ctypes.byref(prob), 1,
                                ctypes.byref(B.gp_solve_opts(nlanczos=10)))
    withp = L.gp_workspace_bytes(B.OP_PCG, ctypes.byref(prob), 1, ctypes.byref(opts))
    assert base > 0 and withp - base >= 4 * 1024 * 50
    # Rank beyond n is taken as n.
    opts.precond_rank = 4000
    big = L.gp_workspace_bytes(B.OP_PCG, ctypes.byref(prob), 1, ctypes.byref(opts))
    opts.precond_rank = 1000
    assert L.gp_workspace_bytes(B.OP_PCG, ctypes.byref(prob), 1, ctypes.byref(opts)) == big
    for bad in (-1, B.MAX_PRECOND_RANK + 1):
        opts.precond_rank = bad
        assert L.gp_workspace_bytes(B.OP_PCG, ctypes.byref(prob), 1, ctypes.byref(opts)) == 0
    opts.precond_rank = 0
    assert L.gp_workspace_bytes(B.OP_NYSTROM, ctypes.byref(prob), 1, ctypes.byref(opts)) == 0
    rank = ctypes.c_int32()
    st = L.gp_nystrom_apply(ctypes.byref(prob), 0, 0.0, 256, 1, 512, None, None, ctypes.byref(rank),
                            1024, 1 << 20, None)
    assert st == B.GP_ERR_ARG and b"k must be" in L.gp_last_error()


def test_workspace_grows_with_problem(L):
    from paper_2503_02259_gb300 import _binding as B
    a = B.gp_problem(256, 1000, 3, 1, B.gp_theta(0.1, 1.0, 0.3))
    b = B.gp_problem(256, 100000, 3, 1, B.gp_theta(0.1, 1.0, 0.3))
    wa = L.gp_workspace_bytes(B.OP_GRAD_MATMUL, ctypes.byref(a), 32, None)
    wb = L.gp_workspace_bytes(B.OP_GRAD_MATMUL, ctypes.byref(b), 32, None)
    assert wb > 10 * wa
    # At least the padded copies of X and V plus two partial planes.
    assert wb >= 4 * 100096 * (4 + 32 + 2 * 32)


@pytest.fixture(scope="module")
def tri(tmp_path_factory):
    d = tmp_path_factory.mktemp("tri")
    src = d / "tri.cpp"
    src.write_text('#include "%s"\n'
                   'extern "C" int eig(double* a, double* b, double* q, int m)'
                   '{ return gp::tridiag_eig_first_row(a, b, q, m) ? 1 : 0; }\n'
                   'extern "C" double quad(const double* al, const double* be, int m, double z2)'
                   '{ double a[64], b[64], q[64]; bool ok; '
                   'double v = gp::lanczos_logquad(al, be, 1, m, z2, a, b, q, &ok); '
                   'return ok ? v : -1e300; }\n'
                   % os.path.join(ROOT, "paper_2503_02259_gb300", "csrc", "tridiag.cuh"))
    so = d / "tri.so"
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", str(src), "-o", str(so)], check=True)
    return ctypes.CDLL(str(so))


@pytest.mark.parametrize("m", [1, 2, 3, 7, 30, 40, 64])
def test_device_eigensolver_host_build_matches_lapack(tri, m):
    rng = np.random.default_rng(m)
    for trial in range(10):
        a = rng.standard_normal(m) * (1 + trial)
        b = rng.standard_normal(max(m - 1, 0))
        if trial % 3 == 0:
            b[::4] *= 1e-10
        A = a.copy()
        Bv = np.append(b, 0.0)
        Q = np.zeros(m)
        vp = ctypes.c_void_p
        assert tri.eig(vp(A.ctypes.data), vp(Bv.ctypes.data), vp(Q.ctypes.data), m)
        if m > 1:
            lam, U = sla.eigh_tridiagonal(a, b)
        else:
            lam, U = a.copy(), np.ones((1, 1))
        idx = np.argsort(A)
        np.testing.assert_allclose(A[idx], lam, atol=1e-13 * max(1, np.abs(lam).max()))
        np.testing.assert_allclose(Q[idx] ** 2, U[0] ** 2, atol=1e-12)


def test_device_gauss_quadrature_host_build_matches_lapack_rule(tri):
    # The device's Gauss rule from Lanczos coefficients, host build, vs the same
    # rule through LAPACK's tridiagonal eigensolver on the same coefficients.
    import oracle as O
    from paper_2503_02259_gb300 import inputs
    X = inputs.points(150, 3, seed=3)
    A = O.khat_dense(X, O.GAUSSIAN, (0.1, 1.0, 0.3))
    z = O.rademacher_probes(150, 1, 9)[:, 0]
    a, b = O.lanczos(A, z, 20)
    bb = np.append(b, 0.0)
    tri.quad.restype = ctypes.c_double
    v = tri.quad(ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(bb.ctypes.data), a.size,
                 ctypes.c_double(150.0))
    ref = O.gauss_quadrature_log(a, b, 150.0)
    assert v == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("d,kind,theta,k", [
    (3, 0, (0.1, 1.0, 0.3), 30),     # the small problem's kernel and SLQ length
    (2, 0, (0.01, 1.0, 0.05), 40),   # the ill-conditioned precision problem's kernel
    (3, 1, (0.05, 1.5, 0.2), 30),    # Matern-3/2 of the product workload
    (8, 0, (0.1, 1.0, 1.2), 40),     # the differentiation problem's kernel (d = 8)
])
def test_device_gauss_quadrature_on_workload_lanczos_matrices(tri, d, kind, theta, k):
    # Lanczos matrices of the workloads' kernels (n = 1500 stand-ins), several
    # probes each: the device's Gauss rule (host build) against LAPACK's, and
    # its exact response to scaling T by c, which adds ||z||^2 log c (the first
    # components sum to one) and must not under- or overflow.
    import oracle as O
    from paper_2503_02259_gb300 import inputs
    n = 1500
    X = inputs.points(n, d, seed=11 + d).astype(np.float64)
    if d == 8:
        X = 0.5 * np.random.default_rng(5).standard_normal((n, d))
    A = O.khat_dense(X, kind, theta)
    Z = O.rademacher_probes(n, 3, 21)
    tri.quad.restype = ctypes.c_double
    vp = ctypes.c_void_p
    for i in range(3):
        a, b = O.lanczos(A, Z[:, i], k)
        bb = np.append(b, 0.0)
        v = tri.quad(vp(a.ctypes.data), vp(bb.ctypes.data), a.size, ctypes.c_double(n))
        ref = O.gauss_quadrature_log(a, b, float(n))
        assert v == pytest.approx(ref, rel=1e-11, abs=1e-9 * n)
        for c in (1e-150, 1e150):
            ac, bc = a * c, np.append(b * c, 0.0)
            vc = tri.quad(vp(ac.ctypes.data), vp(bc.ctypes.data), a.size, ctypes.c_double(n))
            assert vc == pytest.approx(v + n * np.log(c), rel=1e-11, abs=1e-9 * n)
