"""torch.autograd wrappers: eigenpairs of symmetric tridiagonals with a
backward pass through the library's adjoint kernels (mrrr_backward).

    W, Z = eigh_tridiagonal_autograd(d, e)          # d (n,), e (n-1,) or (n,)
    loss = (w * W).sum() + ((C * Z).sum(0) ** 2).sum()
    loss.backward()                                 # d.grad, e.grad

The gradient follows first-order perturbation theory of T = Z diag(W) Z^T
(dbar_j = Tbar(j,j), ebar_j = Tbar(j,j+1) + Tbar(j+1,j) for
Tbar = Z (diag(Wbar) + F o (Z^T Zbar)) Z^T); it is defined for losses that
do not depend on the signs of the columns of Z, and for separated
eigenvalues: gaps at most tau_rel * max|W| are dropped from F (default
api.DEFAULT_TAU_REL = 64 eps, i.e. pairs closer than 64 eps ||T||, which no
FP64 solver can tell apart).
"""
from __future__ import annotations

import torch

from . import api


class EighTridiagonal(torch.autograd.Function):
    """One problem: (d, e) -> (W, Z), all eigenpairs.  With recompute, only
    (d, e) are kept for the backward pass, which solves again (the solver is
    deterministic, so W and Z come out identical)."""

    @staticmethod
    def forward(ctx, d, e, tau_rel=api.DEFAULT_TAU_REL, plan=None, recompute=False):
        W, Z = api.eigh_tridiagonal(d.detach(), e.detach(), plan=plan)
        ctx.tau_rel = float(tau_rel)
        ctx.plan = plan
        ctx.e_numel = e.numel()
        ctx.recompute = bool(recompute)
        ctx.save_for_backward(*((d.detach(), e.detach()) if recompute else (W, Z)))
        return W, Z

    @staticmethod
    def backward(ctx, gW, gZ):
        if ctx.recompute:
            d, e = ctx.saved_tensors
            W, Z = api.eigh_tridiagonal(d, e, plan=ctx.plan)
        else:
            W, Z = ctx.saved_tensors
        n = W.numel()
        layout = api.BatchLayout([n], W.device)
        Zflat = Z.t().contiguous().view(-1)  # column-major storage of Z
        Zb = gZ.t().contiguous().view(-1) if gZ is not None else None
        Wb = gW.contiguous() if gW is not None else None
        dbar, ebar = api.eigh_tridiagonal_backward(W, Zflat, Wb, Zb, layout, tau_rel=ctx.tau_rel, plan=ctx.plan)
        ge = torch.zeros(ctx.e_numel, dtype=dbar.dtype, device=dbar.device)
        m = min(ctx.e_numel, max(n - 1, 0))
        ge[:m] = ebar[:m]
        return dbar[:n], ge, None, None, None


class EighTridiagonalBatched(torch.autograd.Function):
    """A batch packed by an all-eigenpair BatchLayout: (d, e) -> packed (W, Z).
    With recompute, the backward pass solves the batch again instead of
    keeping Z (sum n_p^2 doubles) alive between the passes."""

    @staticmethod
    def forward(ctx, d, e, layout, tau_rel=api.DEFAULT_TAU_REL, plan=None, recompute=False):
        if not layout.all:
            raise ValueError("autograd needs all eigenpairs of every problem")
        W, Z = api.eigh_tridiagonal_batched(d.detach(), e.detach(), layout, plan=plan)
        W = W[:layout.k_total]
        Z = Z[:layout.z_total]
        ctx.layout = layout
        ctx.tau_rel = float(tau_rel)
        ctx.plan = plan
        ctx.d_numel = d.numel()
        ctx.e_numel = e.numel()
        ctx.recompute = bool(recompute)
        ctx.save_for_backward(*((d.detach(), e.detach()) if recompute else (W, Z)))
        return W, Z

    @staticmethod
    def backward(ctx, gW, gZ):
        if ctx.recompute:
            d, e = ctx.saved_tensors
            W, Z = api.eigh_tridiagonal_batched(d, e, ctx.layout, plan=ctx.plan)
            W, Z = W[:ctx.layout.k_total], Z[:ctx.layout.z_total]
        else:
            W, Z = ctx.saved_tensors
        Wb = gW.contiguous() if gW is not None else None
        Zb = gZ.contiguous() if gZ is not None else None
        dbar, ebar = api.eigh_tridiagonal_backward(W, Z, Wb, Zb, ctx.layout, tau_rel=ctx.tau_rel, plan=ctx.plan)
        # d and e may hold more than n_total entries; those get zero gradient
        nt = ctx.layout.n_total
        gd = torch.zeros(ctx.d_numel, dtype=dbar.dtype, device=dbar.device)
        gd[:min(ctx.d_numel, nt)] = dbar[:min(ctx.d_numel, nt)]
        ge = torch.zeros(ctx.e_numel, dtype=dbar.dtype, device=dbar.device)
        m = min(ctx.e_numel, nt)
        ge[:m] = ebar[:m]
        return gd, ge, None, None, None, None


def eigh_tridiagonal_autograd(d: torch.Tensor, e: torch.Tensor, *, tau_rel: float = api.DEFAULT_TAU_REL,
                              plan=None, recompute: bool = False):
    """All eigenpairs (W, Z) of one tridiagonal, differentiable in (d, e)."""
    return EighTridiagonal.apply(d, e, tau_rel, plan, recompute)


def eigh_tridiagonal_batched_autograd(d: torch.Tensor, e: torch.Tensor, layout, *,
                                      tau_rel: float = api.DEFAULT_TAU_REL,
                                      plan=None, recompute: bool = False):
    """Packed all-eigenpair solution of a batch, differentiable in (d, e);
    recompute trades a second solve for not keeping Z between the passes."""
    return EighTridiagonalBatched.apply(d, e, layout, tau_rel, plan, recompute)
