"""Differentiable KKT solve: x = K^{-1} b as a torch.autograd.Function.

Forward factors the KKT matrix assembled from (H values, J values, Sigma,
delta, rho) and solves with refinement; backward is the hand-written
adjoint of the library (ncl_kkt_adjoint), which reuses the same factors:

    g_b = K^{-1} g_x                  (K symmetric)
    dl/dK = -g_b x^T                  folded onto the stored values of
                                      H, J and Sigma (and delta, rho)

so one backward costs one refined solve plus one pass over the pattern.
The gradients of delta and rho are returned when they are passed as
tensors that require a gradient, else None.
"""
from __future__ import annotations

import torch

from .ncl_kkt import KKT


class NclKKTSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kkt: KKT, H_val, J_val, Sigma, b, delta, rho):
        d = delta.detach().cpu().numpy() if torch.is_tensor(delta) else delta
        r = rho.detach().cpu().numpy() if torch.is_tensor(rho) else rho
        if kkt.count == 1 and hasattr(d, "shape") and d.shape:
            d, r = float(d.reshape(-1)[0]), float(r.reshape(-1)[0])
        kkt.factor(H_val.detach(), J_val.detach(), Sigma.detach(), d, r)
        x, info = kkt.solve(b.detach())
        if info.status not in (0,):
            raise RuntimeError(f"KKT solve did not converge (status {info.status})")
        ctx.kkt = kkt
        ctx.generation = kkt.generation
        ctx.scalar_tensors = (torch.is_tensor(delta), torch.is_tensor(rho))
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        kkt = ctx.kkt
        if kkt.generation != ctx.generation:
            raise RuntimeError("the KKT handle was refactored between forward and backward")
        g = kkt.adjoint(x, gx.contiguous())
        gd = gr = None
        if g["scal"] is not None:
            sc = g["scal"].view(-1, 2)
            if ctx.scalar_tensors[0]:
                gd = sc[:, 0].reshape(-1) if kkt.count > 1 else sc[0, 0]
            if ctx.scalar_tensors[1]:
                gr = sc[:, 1].reshape(-1) if kkt.count > 1 else sc[0, 1]
        gd = gd.cpu() if gd is not None else None
        gr = gr.cpu() if gr is not None else None
        return None, g["H"], g["J"], g["Sigma"], g["b"], gd, gr


def kkt_solve(kkt: KKT, H_val, J_val, Sigma, b, delta, rho):
    """x = K^{-1} b, differentiable in H_val, J_val, Sigma, b (and delta,
    rho if given as tensors)."""
    return NclKKTSolve.apply(kkt, H_val, J_val, Sigma, b, delta, rho)
