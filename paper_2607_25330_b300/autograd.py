"""torch.autograd bridge for the PSFD residual (differentiation through the operator).

PhysicsLoss wraps the library's psfd_physics_loss: the physics-informed loss of Eq. loss,
    J = (1/N) sum_a ||r_a||^2 + (lambda_hf / N) sum_a ||w(nu) F3[r_a]||^2,  r = A E - b,
and its gradient (2/N) A^H [r + lambda_hf F3^H (w^2 F3 r)], both computed by the library's
kernels (operator, hand-written adjoint, its own 3-D FFTs, FP64 sums); the backward only
scales the stored gradient.  So J can be differentiated with respect to a predicted field E
without precomputed solutions.  PSFDApply wraps y = A E (psfd_apply, real space) with the
adjoint A^H (psfd_apply with PSFD_ADJOINT) as its backward, for other losses of the residual.

FNOApply wraps the factorised FNO (Sec. 2.1) with its hand-written reverse pass
(fno_forward_train / fno_backward), so that J can be minimised over the network
parameters (Sec. 2.2).
"""
from __future__ import annotations

import torch

from . import psfd


class PSFDApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E: torch.Tensor, plan: "psfd.Plan"):
        ctx.plan = plan
        return plan.apply(E.contiguous())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        # torch's complex convention: for a linear map y = A E the input gradient is A^H g
        return ctx.plan.apply(g.contiguous(), flags=psfd.PSFD_ADJOINT), None


class FNOApply(torch.autograd.Function):
    """E = G_theta(a); params in psfd.FNO_PARAM_NAMES order (CUDA tensors, kernels complex64)."""

    @staticmethod
    def forward(ctx, a: torch.Tensor, trainer: "psfd.FnoTrainer", *params):
        a = a.contiguous()
        ctx.trainer, ctx.a = trainer, a
        ctx.shapes = [(p.shape, p.dtype) for p in params]
        return trainer.forward(a)

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        grads = {n: torch.zeros(s, dtype=dt, device=gE.device)
                 for n, (s, dt) in zip(psfd.FNO_PARAM_NAMES, ctx.shapes)}
        ctx.trainer.backward(ctx.a, gE.to(torch.complex64), grads)
        return (None, None) + tuple(grads[n] for n in psfd.FNO_PARAM_NAMES)


def fno_apply(trainer: "psfd.FnoTrainer", params, a: torch.Tensor) -> torch.Tensor:
    """Differentiable E = G_theta(a); params: dict of CUDA tensors whose pointers the trainer's struct holds."""
    return FNOApply.apply(a, trainer, *[params[n] for n in psfd.FNO_PARAM_NAMES])


class PhysicsLoss(torch.autograd.Function):
    """J = mean over the plan's right-hand sides of Eq. loss (psfd_physics_loss)."""

    @staticmethod
    def forward(ctx, E: torch.Tensor, plan: "psfd.Plan", b: torch.Tensor, lam_hf: float, w0: float, eta_hf: float):
        J, g = plan.physics_loss(E, b, lam_hf, w0, eta_hf, grad=bool(ctx.needs_input_grad[0]))
        ctx.save_for_backward(g if g is not None else torch.empty(0, device=E.device))
        ctx.nrhs = len(J)
        return torch.tensor(float(J.mean()), dtype=torch.float32, device=E.device)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        (g,) = ctx.saved_tensors
        return g * (gJ.to(torch.float32) / ctx.nrhs), None, None, None, None, None


def physics_loss(plan: "psfd.Plan", E: torch.Tensor, b: torch.Tensor, lam_hf: float = 0.1, w0: float = 1.0,
                 eta_hf: float = 1.0) -> torch.Tensor:
    """Eq. loss averaged over the right-hand sides: E, b [nrhs][3][nz][ny][nx] complex64."""
    return PhysicsLoss.apply(E, plan, b, lam_hf, w0, eta_hf)
