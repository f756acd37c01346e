"""Differentiation through the SRT: a torch.autograd.Function whose backward
is the matched adjoint kernel (Algorithm 2 of the paper), and a least-squares
reconstruction driver built on it.

forward(f) = srt_forward(f) (Algorithm 1); backward(g) = srt_adjoint(g).
Because the adjoint is the exact transpose of the forward (same stored
entries), gradients of any loss through this operator are consistent.  That
consistency is what the paper contrasts with approximate GPU adjoints.
"""
from __future__ import annotations

import dataclasses
import math
import os
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


def _data_key(p: torch.Tensor) -> list:
    """Shape, sum and norm of the data in FP64 on the host: a resumed run
    must be fitting the same p."""
    q = p.detach().double().cpu()
    return [list(q.shape), float(q.sum()), float(q.norm())]


def _load_checkpoint(path: str, plan: Plan, reg: float, key: list) -> dict:
    st = torch.load(path, map_location="cpu", weights_only=True)
    want = {"geom": dataclasses.asdict(plan.geom), "reg": float(reg), "data": key}
    for k, v in want.items():
        if st.get(k) != v:
            raise ValueError(f"checkpoint {path} was written for another {k}: "
                             f"{st.get(k)!r} != {v!r}")
    return st


def _save_checkpoint(path: str, state: dict) -> None:
    """Write to a temporary file and rename it over the old one, so that an
    interruption leaves the previous checkpoint whole."""
    tmp = path + ".tmp"
    torch.save(state, tmp)
    os.replace(tmp, path)


def least_squares(plan: Plan, p: torch.Tensor, iters: int = 50, reg: float = 1e-3,
                  f0: torch.Tensor | None = None, lipschitz: float | None = None,
                  checkpoint: str | None = None, every: int = 10) -> LsqResult:
    """Minimise 1/2 ||A f - p||^2 + reg ||grad f||^2 by gradient descent with a
    fixed step 1/L, L = lambda_max(A^T A) + 24 reg (the gradient of the
    difference term is 2 reg D^T D, and D^T D, a 3-D Laplacian, has norm at
    most 12).  Gradients come from autograd through SRTFunction (backward =
    adjoint kernel).

    With ``checkpoint`` a file path, the iterate, the iteration count, the
    losses so far and lambda_max are saved there after every ``every``
    iterations and after the last.  A call that finds the file resumes from
    it instead of starting from f0, and raises ValueError if the file was
    written for another geometry, reg or data.  The products hold no atomics
    and the iterate is saved exactly, so a resumed run computes the same
    iterates as one that was never interrupted."""
    if every < 1:
        raise ValueError("every must be >= 1")
    start, losses, lam = 0, [], lipschitz
    key = _data_key(p) if checkpoint else None
    if checkpoint and os.path.exists(checkpoint):
        st = _load_checkpoint(checkpoint, plan, reg, key)
        start, losses, lam = int(st["iter"]), list(st["losses"]), float(st["lipschitz"])
        f = st["f"].to(plan.device)
    else:
        f = torch.zeros(plan.geom.f_shape, device=plan.device) if f0 is None else f0.clone()
    if lam is None:
        lam = power_lipschitz(plan)
    L = lam + 24.0 * reg
    step = 1.0 / L
    res = LsqResult(f=f, losses=losses, step=step, lipschitz=lam)
    for it in range(start, iters):
        f.requires_grad_(True)
        r = srt(f, plan) - p
        loss = 0.5 * (r * r).sum() + reg * grad_energy(f)
        (g,) = torch.autograd.grad(loss, f)
        res.losses.append(float(loss.detach()))
        with torch.no_grad():
            f = f - step * g
        if checkpoint and ((it + 1) % every == 0 or it + 1 == iters):
            _save_checkpoint(checkpoint, {
                "iter": it + 1, "f": f.detach().cpu(), "losses": list(res.losses),
                "lipschitz": lam, "geom": dataclasses.asdict(plan.geom), "reg": float(reg),
                "data": key})
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
