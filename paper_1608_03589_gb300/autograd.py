"""Differentiable operators and gradient-based reconstruction on the device.

Section 6 writes reconstruction as minimising ||R f - g||^2 (+ a regulariser) through the
normal equations with R* = B.  Here the discrete operators of the C ABI become
``torch.autograd.Function``s whose backward passes are the library's exact Euclidean
transposes (every operator and every gradient runs in the CUDA kernels of libbp.so):

    radon(f)          forward bp_radon,              backward bp_radon_transpose
    backproject(g)    forward bp_backproject_direct  backward bp_backproject_transpose
                      (or the Fourier-path pair with fourier=True)

``tv_reconstruct`` runs plain gradient descent on ||R f - g||^2 + lam TV(f) with a
smoothed isotropic total variation (torch element-wise ops) and a step from a power-
iteration estimate of the Lipschitz constant.  Its state (f, iteration) can be saved with
``torch.save`` and resumed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from .bp import Plan


class _RadonFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, plan: Plan, fourier: bool):
        ctx.plan, ctx.fourier = plan, fourier
        return plan.radon(img.contiguous(), fourier=fourier)

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.radon_transpose(grad.contiguous(), fourier=ctx.fourier), None, None


class _BackprojectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sino, plan: Plan, fourier: bool):
        ctx.plan, ctx.fourier = plan, fourier
        sino = sino.contiguous()
        return plan.backproject_fourier(sino) if fourier else plan.backproject(sino)

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.backproject_transpose(grad.contiguous(), fourier=ctx.fourier), None, None


def radon(img: torch.Tensor, plan: Plan, fourier: bool = False) -> torch.Tensor:
    """Differentiable R (eq "P_theta") of float32 images [..., N, N]."""
    return _RadonFn.apply(img, plan, fourier)


def backproject(sino: torch.Tensor, plan: Plan, fourier: bool = False) -> torch.Tensor:
    """Differentiable R* (eq "bp_app" or eq "bst") of float32 sinograms [..., n_theta, n_det]."""
    return _BackprojectFn.apply(sino, plan, fourier)


def total_variation(f: torch.Tensor, eps: float = 1e-3) -> torch.Tensor:
    """Smoothed isotropic TV: sum sqrt(dx^2 + dy^2 + eps^2) with forward differences."""
    dx = torch.diff(f, dim=-1, append=f[..., -1:])
    dy = torch.diff(f, dim=-2, append=f[..., -1:, :])
    return torch.sqrt(dx * dx + dy * dy + eps * eps).sum()


def lipschitz_estimate(plan: Plan, shape, device, iters: int = 12, fourier: bool = False) -> float:
    """Largest eigenvalue of R^T R by power iteration (kernels only)."""
    v = torch.randn(shape, device=device, generator=torch.Generator(device=device).manual_seed(0))
    lam = 0.0
    for _ in range(iters):
        v = v / v.norm()
        w = plan.radon_transpose(plan.radon(v, fourier=fourier), fourier=fourier)
        lam = float((v * w).sum())
        v = w
    return lam


@dataclass
class TVState:
    f: torch.Tensor
    iteration: int = 0
    losses: list = field(default_factory=list)


def tv_reconstruct(g: torch.Tensor, plan: Plan, iters: int = 50, lam: float = 1e-3, eps: float = 1e-3,
                   step: float | None = None, fourier: bool = False, state: TVState | None = None) -> TVState:
    """Gradient descent on ||R f - g||^2 + lam TV(f) for sinograms g [..., n_theta, n_det].

    Pass a previous ``state`` to resume; ``state`` is what ``torch.save`` should store.
    """
    batch_shape = g.shape[:-2]
    if state is None:
        state = TVState(f=torch.zeros((*batch_shape, plan.N, plan.N), dtype=torch.float32, device=g.device))
    if step is None:
        L = 2.0 * lipschitz_estimate(plan, (*batch_shape, plan.N, plan.N), g.device, fourier=fourier)
        L += lam * 8.0 / eps
        step = 1.0 / L
    f = state.f.detach().clone()
    for _ in range(iters):
        f.requires_grad_(True)
        r = radon(f, plan, fourier) - g
        loss = (r * r).sum() + lam * total_variation(f, eps)
        (grad,) = torch.autograd.grad(loss, f)
        with torch.no_grad():
            f = f - step * grad
        state.losses.append(float(loss.detach()))
        state.iteration += 1
    state.f = f.detach()
    return state
