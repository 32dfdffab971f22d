"""torch.autograd bridge for the PSFD residual (differentiation through the operator).

PSFDApply wraps y = A E (psfd_apply, real space) with the hand-written adjoint
E_bar = A^H y_bar (psfd_apply with PSFD_ADJOINT) as its backward, so that the
physics-informed loss of Eq. loss,
    J = (1/N) sum_a ||r_a||^2 + (lambda_hf / N) sum_a ||w(nu) F3[r_a]||^2,  r = A E - b,
can be differentiated with respect to a predicted field E without precomputed
solutions.  Both directions run in the library's kernels; torch only holds the
tensors (the loss reductions and F3 of the penalty term are torch GPU ops).
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
