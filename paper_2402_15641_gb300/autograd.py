"""Differentiation through the SRT: a torch.autograd.Function whose backward
is the matched adjoint kernel (Algorithm 2 of the paper), and a least-squares
reconstruction driver built on it.

forward(f) = srt_forward(f) (Algorithm 1); backward(g) = srt_adjoint(g).
Because the adjoint is the exact transpose of the forward (same stored
entries), gradients of any loss through this operator are consistent.  That
consistency is what the paper contrasts with approximate GPU adjoints.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from .srt import Plan


class SRTFunction(torch.autograd.Function):
    """y = A f with dy -> A^T dy, on the plan's CUDA kernels."""

    @staticmethod
    def forward(ctx, f: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.forward(f.contiguous())

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        return ctx.plan.adjoint(grad.contiguous()), None


def srt(f: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable forward transform."""
    return SRTFunction.apply(f, plan)


class SRTAdjointFunction(torch.autograd.Function):
    """f = A^T p with df -> A df (the adjoint of the adjoint)."""

    @staticmethod
    def forward(ctx, p: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.adjoint(p.contiguous())

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        return ctx.plan.forward(grad.contiguous()), None


def srt_adjoint(p: torch.Tensor, plan: Plan) -> torch.Tensor:
    return SRTAdjointFunction.apply(p, plan)


def grad_energy(f: torch.Tensor) -> torch.Tensor:
    """||grad f||^2 with forward differences along x, y and z over interior
    pairs only (no wrap-around)."""
    dx = f[..., 1:, :, :] - f[..., :-1, :, :]
    dy = f[..., :, 1:, :] - f[..., :, :-1, :]
    dz = f[..., :, :, 1:] - f[..., :, :, :-1]
    return (dx * dx).sum() + (dy * dy).sum() + (dz * dz).sum()


def power_lipschitz(plan: Plan, iters: int = 20, seed: int = 2) -> float:
    """Largest eigenvalue of A^T A by power iteration from a seeded start."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.randn(plan.geom.f_shape, generator=g).to(plan.device)
    v /= v.norm()
    lam = 0.0
    for _ in range(iters):
        w = plan.adjoint(plan.forward(v))
        lam = float(torch.dot(v.flatten().double(), w.flatten().double()))
        v = w / w.norm()
    return lam


@dataclass
class LsqResult:
    f: torch.Tensor
    losses: list = field(default_factory=list)
    step: float = 0.0
    lipschitz: float = 0.0


def least_squares(plan: Plan, p: torch.Tensor, iters: int = 50, reg: float = 1e-3,
                  f0: torch.Tensor | None = None, lipschitz: float | None = None) -> LsqResult:
    """Minimise 1/2 ||A f - p||^2 + reg ||grad f||^2 by gradient descent with a
    fixed step 1/L, L = lambda_max(A^T A) + 24 reg (the gradient of the
    difference term is 2 reg D^T D, and D^T D, a 3-D Laplacian, has norm at
    most 12).  Gradients come from autograd through SRTFunction (backward =
    adjoint kernel)."""
    f = torch.zeros(plan.geom.f_shape, device=plan.device) if f0 is None else f0.clone()
    lam = power_lipschitz(plan) if lipschitz is None else lipschitz
    L = lam + 24.0 * reg
    step = 1.0 / L
    res = LsqResult(f=f, step=step, lipschitz=lam)
    for _ in range(iters):
        f.requires_grad_(True)
        r = srt(f, plan) - p
        loss = 0.5 * (r * r).sum() + reg * grad_energy(f)
        (g,) = torch.autograd.grad(loss, f)
        res.losses.append(float(loss))
        with torch.no_grad():
            f = f - step * g
    res.f = f.detach()
    with torch.no_grad():
        r = plan.forward(res.f) - p
        res.losses.append(float(0.5 * (r * r).sum() + reg * grad_energy(res.f)))
    return res


def noisy_data(plan: Plan, f_true: torch.Tensor, level: float = 0.01, seed: int = 1):
    """p = A f + noise with sigma = level * ||A f|| / sqrt(numel p)."""
    clean = plan.forward(f_true)
    sigma = level * float(clean.norm()) / math.sqrt(clean.numel())
    g = torch.Generator(device="cpu").manual_seed(seed)
    noise = torch.randn(clean.shape, generator=g).to(clean.device) * sigma
    return clean + noise, sigma
