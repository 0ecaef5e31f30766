"""Python calls with the names of the C ABI, on torch CUDA tensors.

Each function validates shapes, allocates its outputs and the library's
workspace with torch on the input's device, and calls the C entry point on
torch's current stream.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int32

import torch

from . import _binding as B
from ._binding import check, lib


def _stream(dev) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    return t.contiguous()


def problem(X: torch.Tensor, kernel: int, theta, ls=None) -> tuple[B.gp_problem, torch.Tensor]:
    """gp_problem for device points X (n, d) float32 and theta = (s, f, l); ls:
    optional d per-dimension length-scales (theta's l is then unused)."""
    X = _f32(X, "X")
    if X.dim() != 2:
        raise ValueError("X must be (n, d)")
    s, f, l = (float(v) for v in theta)
    p = B.gp_problem(X.data_ptr(), X.shape[0], X.shape[1], int(kernel), B.gp_theta(s, f, l))
    if ls is not None:
        if len(ls) != X.shape[1]:
            raise ValueError("ls must have d entries")
        arr = (ctypes.c_double * len(ls))(*(float(v) for v in ls))
        p.ls = ctypes.cast(arr, ctypes.c_void_p)
        p._ls_keep = arr   # the host array lives as long as the struct
    return p, X


def solve_opts(nprobe: int = 0, nlanczos: int = 30, cg_maxit: int = 0, cg_rtol: float = 1e-8,
               seed: int = 0, prec: int = B.PREC_FP32, refine_rtol: float = 0.0,
               probes: torch.Tensor | None = None, refine_maxit: int = 0,
               slq_prec: int = B.PREC_FP32,
               refine_residual: int = B.RESIDUAL_PAIR, precond_rank: int = 0,
               precond_tol: float = 0.0) -> B.gp_solve_opts:
    """gp_solve_opts; slq_prec is the arithmetic of the SLQ Lanczos products
    (B.PREC_SAME: the same as prec); refine_residual the arithmetic of the
    refinement's outer residual (B.RESIDUAL_PAIR or B.RESIDUAL_FP64);
    precond_rank > 0 selects the Nystrom preconditioner of that rank for the
    solves (precond_tol: its early stop, relative to f^2)."""
    o = B.gp_solve_opts(int(nprobe), int(nlanczos), int(cg_maxit), int(prec), float(cg_rtol),
                        float(refine_rtol), int(seed) & (2**64 - 1),
                        0 if probes is None else probes.data_ptr(), int(refine_maxit),
                        int(slq_prec), int(refine_residual), int(precond_rank),
                        float(precond_tol))
    o._probes_keep = probes   # the struct holds only the address: keep the tensor alive with it
    return o


def workspace(op: int, prob: B.gp_problem, w: int, opts: B.gp_solve_opts | None, device) -> torch.Tensor:
    nbytes = lib().gp_workspace_bytes(op, byref(prob), int(w), None if opts is None else byref(opts))
    if nbytes == 0:
        raise B.GPError(B.GP_ERR_ARG, "gp_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    if ws.data_ptr() % 256:
        raise RuntimeError("workspace allocation is not 256-byte aligned")
    return ws


def gp_kernel_matmul(X, V, kernel, theta, prec=B.PREC_FP32, ws=None, ls=None) -> torch.Tensor:
    """Y = Kh V on the device."""
    prob, X = problem(X, kernel, theta, ls)
    V = _f32(V, "V")
    if V.dim() == 1:
        V = V[:, None]
    n, w = V.shape
    if n != X.shape[0]:
        raise ValueError("V must have n rows")
    Y = torch.empty_like(V)
    if ws is None:
        ws = workspace(B.OP_MATMUL, prob, w, B.gp_solve_opts(prec=prec) if prec else None, X.device)
    check(lib().gp_kernel_matmul(byref(prob), _ptr(V), w, _ptr(Y), int(prec), _ptr(ws), ws.numel(),
                                 _stream(X.device)), "gp_kernel_matmul")
    return Y


def gp_kernel_grad_matmul(X, V, kernel, theta, ws=None):
    """(Kh V, dKh/df V, dKh/dl V) from one fused pass (dKh/ds V = V)."""
    prob, X = problem(X, kernel, theta)
    V = _f32(V, "V")
    if V.dim() == 1:
        V = V[:, None]
    n, w = V.shape
    Y = torch.empty_like(V)
    dYf = torch.empty_like(V)
    dYl = torch.empty_like(V)
    if ws is None:
        ws = workspace(B.OP_GRAD_MATMUL, prob, w, None, X.device)
    check(lib().gp_kernel_grad_matmul(byref(prob), _ptr(V), w, _ptr(Y), _ptr(dYf), _ptr(dYl),
                                      B.PREC_FP32, _ptr(ws), ws.numel(), _stream(X.device)),
          "gp_kernel_grad_matmul")
    return Y, dYf, dYl


def gp_pcg_solve(X, Bm, kernel, theta, opts: B.gp_solve_opts, raise_not_converged=True, ws=None,
                 ls=None):
    """Column-wise CG: returns (Xsol, iters (w,), relres (w,), status)."""
    prob, X = problem(X, kernel, theta, ls)
    Bm = _f32(Bm, "B")
    if Bm.dim() == 1:
        Bm = Bm[:, None]
    n, w = Bm.shape
    Xsol = torch.empty_like(Bm)
    iters = (c_int32 * w)()
    relres = (c_double * w)()
    if ws is None:
        ws = workspace(B.OP_PCG, prob, w, opts, X.device)
    st = lib().gp_pcg_solve(byref(prob), _ptr(Bm), w, _ptr(Xsol), byref(opts), iters, relres,
                            _ptr(ws), ws.numel(), _stream(X.device))
    if st != B.GP_OK and not (st == B.GP_ERR_NOT_CONVERGED and not raise_not_converged):
        check(st, "gp_pcg_solve")
    return Xsol, list(iters), list(relres), st


def gp_nystrom_apply(X, V, kernel, theta, k: int, tol: float = 0.0, want_L: bool = False,
                     ls=None, ws=None):
    """Nystrom preconditioner of rank <= k: returns (Z = M^-1 V (n, w), L (n, rank)
    float32 or None, pivots (rank,), rank)."""
    prob, X = problem(X, kernel, theta, ls)
    V = _f32(V, "V")
    if V.dim() == 1:
        V = V[:, None]
    n, w = V.shape
    if n != X.shape[0]:
        raise ValueError("V must have n rows")
    Z = torch.empty_like(V)
    kk = min(int(k), n)
    Lc = torch.empty((kk, n), dtype=torch.float32, device=X.device) if want_L else None
    piv = (ctypes.c_int64 * max(kk, 1))()
    rank = c_int32()
    if ws is None:
        ws = workspace(B.OP_NYSTROM, prob, w, solve_opts(precond_rank=k), X.device)
    check(lib().gp_nystrom_apply(byref(prob), int(k), float(tol), _ptr(V), w, _ptr(Z), _ptr(Lc),
                                 piv, byref(rank), _ptr(ws), ws.numel(), _stream(X.device)),
          "gp_nystrom_apply")
    r = rank.value
    L = None if Lc is None else Lc[:r].t()
    return Z, L, list(piv)[:r], r


def gp_pcg_solve_refined(X, Bm, kernel, theta, opts: B.gp_solve_opts, raise_not_converged=True,
                         ws=None):
    """Mixed-precision iterative refinement with an FP64 solution:
    returns (X64 (n, w) float64, total inner iterations (w,), final relres (w,), status)."""
    prob, X = problem(X, kernel, theta)
    Bm = _f32(Bm, "B")
    if Bm.dim() == 1:
        Bm = Bm[:, None]
    n, w = Bm.shape
    X64 = torch.empty((n, w), dtype=torch.float64, device=X.device)
    iters = (c_int32 * w)()
    relres = (c_double * w)()
    if ws is None:
        ws = workspace(B.OP_PCG, prob, w, opts, X.device)
    st = lib().gp_pcg_solve_refined(byref(prob), _ptr(Bm), w, _ptr(X64), byref(opts), iters, relres,
                                    _ptr(ws), ws.numel(), _stream(X.device))
    if st != B.GP_OK and not (st == B.GP_ERR_NOT_CONVERGED and not raise_not_converged):
        check(st, "gp_pcg_solve_refined")
    return X64, list(iters), list(relres), st


def gp_true_residual(X, Bm, Xsol, kernel, theta, ws=None) -> list:
    """||B_c - Kh X_c|| / ||B_c|| per column, FP64 entries and sums."""
    prob, X = problem(X, kernel, theta)
    Bm = _f32(Bm, "B")
    Xsol = _f32(Xsol, "Xsol")
    if Bm.dim() == 1:
        Bm = Bm[:, None]
    if Xsol.dim() == 1:
        Xsol = Xsol[:, None]
    n, w = Bm.shape
    if Xsol.shape != (n, w):
        raise ValueError("B and Xsol must have the same shape")
    relres = (c_double * w)()
    if ws is None:
        ws = workspace(B.OP_RESIDUAL, prob, w, None, X.device)
    check(lib().gp_true_residual(byref(prob), _ptr(Bm), _ptr(Xsol), w, relres, _ptr(ws), ws.numel(),
                                 _stream(X.device)), "gp_true_residual")
    return list(relres)


def gp_residual_rows(X, Bm, X64, kernel, theta, rows=None, m=None, arith=B.RESIDUAL_PAIR,
                     ws=None, want_rows=True):
    """Residual rows R = B[rows] - (Kh X64)[rows] (FP64, (m, w)) and the
    per-column ||R_c|| / ||B_rows,c||, in the arithmetic `arith`.  rows: device
    int64 indices, or None for the first m rows (all n when m is None)."""
    prob, X = problem(X, kernel, theta)
    Bm = _f32(Bm, "B")
    if Bm.dim() == 1:
        Bm = Bm[:, None]
    if not X64.is_cuda or X64.dtype != torch.float64:
        raise ValueError("X64 must be a float64 CUDA tensor")
    X64 = X64.contiguous()
    if X64.dim() == 1:
        X64 = X64[:, None]
    n, w = Bm.shape
    if X64.shape != (n, w):
        raise ValueError("B and X64 must have the same shape")
    if rows is not None:
        if not rows.is_cuda or rows.dtype != torch.int64:
            raise ValueError("rows must be an int64 CUDA tensor")
        rows = rows.contiguous()
        m = rows.numel()
    elif m is None:
        m = n
    R = torch.empty((m, w), dtype=torch.float64, device=X.device) if want_rows else None
    relres = (c_double * w)()
    if ws is None:
        ws = workspace(B.OP_RESIDUAL, prob, w, None, X.device)
    check(lib().gp_residual_rows(byref(prob), _ptr(Bm), _ptr(X64), w, _ptr(rows), int(m),
                                 int(arith), _ptr(R), relres, _ptr(ws), ws.numel(),
                                 _stream(X.device)), "gp_residual_rows")
    return R, list(relres)


def gp_slq_logdet(X, kernel, theta, opts: B.gp_solve_opts, ws=None):
    prob, X = problem(X, kernel, theta)
    ld = c_double()
    se = c_double()
    if ws is None:
        ws = workspace(B.OP_SLQ, prob, 0, opts, X.device)
    check(lib().gp_slq_logdet(byref(prob), byref(opts), byref(ld), byref(se), _ptr(ws), ws.numel(),
                              _stream(X.device)), "gp_slq_logdet")
    return ld.value, se.value


def gp_loss_and_grad(X, y, kernel, theta, opts: B.gp_solve_opts, ws=None, ls=None):
    """(loss, [dL/ds, dL/df, dL/dl], info dict); with per-dimension length-scales
    ls the gradient is [dL/ds, dL/df, dL/dl_1, ..., dL/dl_d]."""
    prob, X = problem(X, kernel, theta, ls)
    y = _f32(y, "y").reshape(-1)
    loss = c_double()
    grad = (c_double * (3 if ls is None else 2 + X.shape[1]))()
    info = B.gp_loss_info()
    if ws is None:
        ws = workspace(B.OP_LOSS_GRAD, prob, 0, opts, X.device)
    check(lib().gp_loss_and_grad(byref(prob), _ptr(y), byref(opts), byref(loss), grad, byref(info),
                                 _ptr(ws), ws.numel(), _stream(X.device)), "gp_loss_and_grad")
    return loss.value, list(grad), info.as_dict()


def gp_loss_and_grad_batch(Xs, ys, kernels, thetas, opts_list, raise_not_converged=True):
    """gp_loss_and_grad for several problems at once (one grouped product launch
    per solver step): returns ([loss], [[dL/ds, dL/df, dL/dl]], [info], [status])."""
    count = len(Xs)
    probs = (B.gp_problem * count)()
    keep = []
    for k in range(count):
        p, X = problem(Xs[k], kernels[k], thetas[k])
        probs[k] = p
        keep.append(X)
    yv = [_f32(y, "y").reshape(-1) for y in ys]
    yp = (ctypes.c_void_p * count)(*[y.data_ptr() for y in yv])
    opts = (B.gp_solve_opts * count)(*opts_list)
    wss = [workspace(B.OP_LOSS_GRAD_BATCH, probs[k], 0, opts[k], keep[k].device)
           for k in range(count)]
    wsp = (ctypes.c_void_p * count)(*[w.data_ptr() for w in wss])
    wsb = (ctypes.c_size_t * count)(*[w.numel() for w in wss])
    loss = (c_double * count)()
    grad = (c_double * (3 * count))()
    info = (B.gp_loss_info * count)()
    status = (c_int32 * count)()
    st = lib().gp_loss_and_grad_batch(count, probs, yp, opts, loss, grad, info, status, wsp, wsb,
                                      _stream(keep[0].device))
    if st != B.GP_OK and not (st == B.GP_ERR_NOT_CONVERGED and not raise_not_converged):
        check(st, "gp_loss_and_grad_batch")
    return (list(loss), [list(grad[3 * k:3 * k + 3]) for k in range(count)],
            [i.as_dict() for i in info], list(status))


def gp_nll_forward(X, y, kernel, theta, opts: B.gp_solve_opts, ls=None):
    """(loss, W = Kh^-1 [y | Z] (n, 1 + p), info)."""
    prob, X = problem(X, kernel, theta, ls)
    y = _f32(y, "y").reshape(-1)
    W = torch.empty((X.shape[0], 1 + opts.nprobe), dtype=torch.float32, device=X.device)
    loss = c_double()
    info = B.gp_loss_info()
    ws = workspace(B.OP_LOSS_GRAD, prob, 0, opts, X.device)
    check(lib().gp_nll_forward(byref(prob), _ptr(y), byref(opts), _ptr(W), byref(loss), byref(info),
                               _ptr(ws), ws.numel(), _stream(X.device)), "gp_nll_forward")
    return loss.value, W, info.as_dict()


def gp_nll_backward(X, W, kernel, theta, opts: B.gp_solve_opts, ls=None):
    """[dL/ds, dL/df, dL/dl] from the forward's W (probes regenerated, not stored);
    [dL/ds, dL/df, dL/dl_1, ..., dL/dl_d] with per-dimension length-scales ls."""
    prob, X = problem(X, kernel, theta, ls)
    W = _f32(W, "W")
    grad = (c_double * (3 if ls is None else 2 + X.shape[1]))()
    info = B.gp_loss_info()
    ws = workspace(B.OP_LOSS_GRAD, prob, 0, opts, X.device)
    check(lib().gp_nll_backward(byref(prob), byref(opts), _ptr(W), grad, byref(info), _ptr(ws),
                                ws.numel(), _stream(X.device)), "gp_nll_backward")
    return list(grad), info.as_dict()


def gp_predict_mean(X, alpha, Xstar, kernel, theta, prec=B.PREC_FP32, ws=None, ls=None):
    """mu = f^2 K(X*, X) alpha."""
    prob, X = problem(X, kernel, theta, ls)
    alpha = _f32(alpha, "alpha").reshape(-1)
    Xstar = _f32(Xstar, "Xstar")
    m = Xstar.shape[0]
    mu = torch.empty(m, dtype=torch.float32, device=X.device)
    if ws is None:
        ws = workspace(B.OP_PREDICT, prob, m, None, X.device)
    check(lib().gp_predict_mean(byref(prob), _ptr(alpha), _ptr(Xstar), m, _ptr(mu), int(prec),
                                _ptr(ws), ws.numel(), _stream(X.device)), "gp_predict_mean")
    return mu


def gp_predict_var(X, Xstar, kernel, theta, opts: B.gp_solve_opts, raise_not_converged=True,
                   ws=None, ls=None):
    """Posterior variance of the noise-free test outputs at Xstar: returns
    (var (m,), largest CG iteration count, largest final relres, status)."""
    prob, X = problem(X, kernel, theta, ls)
    Xstar = _f32(Xstar, "Xstar")
    m = Xstar.shape[0]
    var = torch.empty(m, dtype=torch.float32, device=X.device)
    it = c_int32()
    rel = c_double()
    if ws is None:
        ws = workspace(B.OP_PREDICT_VAR, prob, m, opts, X.device)
    st = lib().gp_predict_var(byref(prob), _ptr(Xstar), m, _ptr(var), byref(opts), byref(it),
                              byref(rel), _ptr(ws), ws.numel(), _stream(X.device))
    if st != B.GP_OK and not (st == B.GP_ERR_NOT_CONVERGED and not raise_not_converged):
        check(st, "gp_predict_var")
    return var, it.value, rel.value, st


def gp_generate_probes(n: int, p: int, seed: int, device="cuda") -> torch.Tensor:
    Z = torch.empty((n, p), dtype=torch.float32, device=device)
    check(lib().gp_generate_probes(n, p, int(seed) & (2**64 - 1), _ptr(Z), p,
                                   _stream(Z.device)), "gp_generate_probes")
    return Z
