"""torch.autograd bridge for the PSFD residual (differentiation through the operator).

PSFDApply wraps y = A E (psfd_apply, real space) with the hand-written adjoint
E_bar = A^H y_bar (psfd_apply with PSFD_ADJOINT) as its backward, so that the
physics-informed loss of Eq. loss,
    J = (1/N) sum_a ||r_a||^2 + (lambda_hf / N) sum_a ||w(nu) F3[r_a]||^2,  r = A E - b,
can be differentiated with respect to a predicted field E without precomputed
solutions.  Both directions run in the library's kernels; torch only holds the
tensors (the loss reductions and F3 of the penalty term are torch GPU ops).

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


def frequency_weight(nz: int, ny: int, nx: int, w0: float = 1.0, eta_hf: float = 1.0, device="cuda"):
    f = lambda n: torch.fft.fftfreq(n, device=device, dtype=torch.float32)
    nu = torch.sqrt(f(nz)[:, None, None] ** 2 + f(ny)[None, :, None] ** 2 + f(nx)[None, None, :] ** 2)
    return w0 + eta_hf * nu


def physics_loss(plan: "psfd.Plan", E: torch.Tensor, b: torch.Tensor, lam_hf: float = 0.1, w0: float = 1.0,
                 eta_hf: float = 1.0) -> torch.Tensor:
    """Eq. loss averaged over the right-hand sides: E, b [nrhs][3][nz][ny][nx] complex64."""
    r = PSFDApply.apply(E, plan) - b
    nz, ny, nx = r.shape[-3:]
    N = nz * ny * nx
    wgt = frequency_weight(nz, ny, nx, w0, eta_hf, device=r.device)
    R3 = torch.fft.fftn(r, dim=(-3, -2, -1), norm="ortho")
    per = (r.abs() ** 2).sum(dim=(-4, -3, -2, -1)) / N + lam_hf * ((wgt * R3.abs()) ** 2).sum(dim=(-4, -3, -2, -1)) / N
    return per.mean()
