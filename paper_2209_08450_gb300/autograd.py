"""Differentiable projector/backprojector pair and least-squares reconstruction.

The LineRec backprojection (Sec. 2.2 / Sec. 3 of the TomocuPy paper) and its
exact transpose, the Radon projector, become a torch.autograd.Function pair:
the backward of each is the other's hand-written CUDA kernel.  Both operators
are linear, so nothing is saved for backward (recomputation instead of stored
intermediates).  Iterative reconstruction is named as future work in the
paper's outlook (Sec. 5); here it is plain gradient descent on
||P x - y||^2.
"""
from __future__ import annotations

import numpy as np
import torch

from . import backproject, project


class Project(torch.autograd.Function):
    """y = P x: vol [nz][n][n] -> sino [nz][ntheta][ndet]; backward is P^T."""

    @staticmethod
    def forward(ctx, vol, theta, center, ndet):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        ctx.theta, ctx.center, ctx.n = th, float(center), vol.shape[-1]
        return project(vol.contiguous(), th, center, ndet)

    @staticmethod
    def backward(ctx, g):
        return backproject(g.contiguous(), ctx.theta, ctx.center, n=ctx.n), None, None, None


class Backproject(torch.autograd.Function):
    """x = P^T y: sino [nz][ntheta][ndet] -> vol [nz][n][n]; backward is P."""

    @staticmethod
    def forward(ctx, sino, theta, center, n):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        ctx.theta, ctx.center, ctx.ndet = th, float(center), sino.shape[-1]
        return backproject(sino.contiguous(), th, center, n=n)

    @staticmethod
    def backward(ctx, g):
        return project(g.contiguous(), ctx.theta, ctx.center, ndet=ctx.ndet), None, None, None


def radon(vol: torch.Tensor, theta, center: float, ndet: int) -> torch.Tensor:
    return Project.apply(vol, theta, center, ndet)


def radon_t(sino: torch.Tensor, theta, center: float, n: int) -> torch.Tensor:
    return Backproject.apply(sino, theta, center, n)


def operator_norm_sq(shape, theta, center: float, ndet: int, iters: int = 20, seed: int = 0,
                     device="cuda") -> float:
    """||P||^2 by power iteration on P^T P (every product is a CUDA kernel)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn(shape, generator=g, device=device)
    x /= x.norm()
    lam = 0.0
    for _ in range(iters):
        y = backproject(project(x, theta, center, ndet), theta, center, n=shape[-1])
        lam = float(y.norm())
        x = y / lam
    return lam


def lsq_gradient_descent(y: torch.Tensor, theta, center: float, n: int, iters: int = 50,
                         step: float | None = None, x0: torch.Tensor | None = None,
                         callback=None) -> torch.Tensor:
    """Minimise L(x) = ||P x - y||^2 by gradient descent with autograd.

    The gradient 2 P^T (P x - y) comes from Project.backward (the
    backprojection kernel).  Default step 1/L with L = 2 ||P||^2."""
    ndet = y.shape[-1]
    x = (torch.zeros((y.shape[0], n, n), device=y.device) if x0 is None else x0.clone()).requires_grad_(True)
    if step is None:
        step = 1.0 / (2.0 * operator_norm_sq((1, n, n), theta, center, ndet, device=y.device))
    for it in range(iters):
        loss = torch.sum((radon(x, theta, center, ndet) - y) ** 2)
        (gx,) = torch.autograd.grad(loss, x)
        with torch.no_grad():
            x -= step * gx
        if callback is not None:
            callback(it, float(loss.detach()))
    return x.detach()
