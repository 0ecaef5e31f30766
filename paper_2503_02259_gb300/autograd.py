"""L(Theta) as a torch.autograd.Function with a hand-written backward.

The paper computes dL/dtheta with hand-coded formulas rather than automatic
differentiation (§Statement of Need, third contribution; the gradient equation
of §Gaussian Processes).  Here the forward runs the block CG on [y | Z] and SLQ
(gp_nll_forward) and keeps only W = Kh^-1 [y | Z]; the backward regenerates the
same probes Z from the seed instead of storing them and runs one fused
derivative product (gp_nll_backward).  With ``recompute=True`` the forward
keeps nothing n-sized and the backward re-solves for W first.  ``prec`` and
``slq_prec`` choose the arithmetic of the CG and of the Lanczos products (the
derivative product of the backward is FP32).  ``theta`` holds (s, f, l), or
(s, f, l_1, ..., l_d) for per-dimension length-scales, whose backward is the
fused contraction of the entries and their d derivatives (no derivative
product).  With ``precond_rank > 0`` the loss is Eq. 1 / Eq. 2 with the
Nystrom preconditioner (isotropic l): the forward runs the whole
gp_loss_and_grad call (the preconditioned gradient needs the factor's
derivative, built in the same pass) and keeps only the gradient's three
numbers, which the backward scales.
"""
from __future__ import annotations

import torch

from . import api
from ._binding import PREC_FP32


class GPNegLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, X, y, kernel, nprobe, nlanczos, cg_rtol, seed, cg_maxit, recompute,
                prec, slq_prec, precond_rank, precond_tol):
        vals = [float(v) for v in theta.detach().cpu().tolist()]
        d = X.shape[1]
        if len(vals) == 3:
            th, ls = vals, None
        elif len(vals) == 2 + d:
            th, ls = [vals[0], vals[1], 1.0], vals[2:]
        else:
            raise ValueError("theta must hold (s, f, l) or (s, f, l_1..l_d)")
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        if precond_rank > 0:
            if ls is not None:
                raise ValueError("the preconditioned loss takes an isotropic length-scale")
            opts = api.solve_opts(nprobe=nprobe, nlanczos=nlanczos, cg_rtol=cg_rtol, seed=seed,
                                  cg_maxit=cg_maxit, prec=prec, slq_prec=slq_prec,
                                  precond_rank=precond_rank, precond_tol=precond_tol)
            loss, grad, info = api.gp_loss_and_grad(X, y, kernel, th, opts)
            ctx.grad = grad
            ctx.info = info
            ctx.save_for_backward()
            return theta.new_tensor(loss)
        ctx.grad = None
        opts = api.solve_opts(nprobe=nprobe, nlanczos=nlanczos, cg_rtol=cg_rtol, seed=seed,
                              cg_maxit=cg_maxit, prec=prec, slq_prec=slq_prec)
        loss, W, info = api.gp_nll_forward(X, y, kernel, th, opts, ls=ls)
        ctx.cfg = (kernel, th, ls, nprobe, nlanczos, cg_rtol, seed, cg_maxit, recompute, prec,
                   slq_prec)
        ctx.info = info
        ctx.save_for_backward(X, y, None if recompute else W)
        return theta.new_tensor(loss)

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.grad is not None:
            g = torch.tensor(ctx.grad, dtype=ctx.theta_dtype, device=ctx.theta_device) * grad_out.to(
                device=ctx.theta_device, dtype=ctx.theta_dtype)
            return (g,) + (None,) * 13
        X, y, W = ctx.saved_tensors
        (kernel, th, ls, nprobe, nlanczos, cg_rtol, seed, cg_maxit, recompute, prec,
         slq_prec) = ctx.cfg
        opts = api.solve_opts(nprobe=nprobe, nlanczos=nlanczos, cg_rtol=cg_rtol, seed=seed,
                              cg_maxit=cg_maxit, prec=prec, slq_prec=slq_prec)
        if W is None:
            _, W, _ = api.gp_nll_forward(X, y, kernel, th, opts, ls=ls)
        grad, _ = api.gp_nll_backward(X, W, kernel, th, opts, ls=ls)
        g = torch.tensor(grad, dtype=ctx.theta_dtype, device=ctx.theta_device) * grad_out.to(
            device=ctx.theta_device, dtype=ctx.theta_dtype)
        return (g,) + (None,) * 13


def neg_log_likelihood(theta: torch.Tensor, X: torch.Tensor, y: torch.Tensor, kernel: int,
                       nprobe: int = 16, nlanczos: int = 30, cg_rtol: float = 1e-6, seed: int = 0,
                       cg_maxit: int = 0, recompute: bool = False, prec: int = PREC_FP32,
                       slq_prec: int = PREC_FP32, precond_rank: int = 0,
                       precond_tol: float = 0.0) -> torch.Tensor:
    """L(theta) with theta = (s, f, l), or (s, f, l_1..l_d) for per-dimension
    length-scales; differentiable in theta.  precond_rank > 0: Eq. 1 / Eq. 2
    with the Nystrom preconditioner of that rank (Gaussian probes from seed)."""
    return GPNegLogLik.apply(theta, X, y, kernel, nprobe, nlanczos, cg_rtol, seed, cg_maxit, recompute,
                             prec, slq_prec, precond_rank, precond_tol)
