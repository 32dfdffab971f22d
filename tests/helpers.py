"""Shared test set-up: the same seeded inputs for the oracle and the CUDA library."""
import numpy as np
import torch

from paper_2607_25330_b300 import inputs as I


def problem(nx, ny, nz, theta=6.0, phi=0.0, pols=(0,), cap=True, dx=2.0, dz=2.0, **kw):
    pml = kw.pop("pml_planes", I.default_pml(nz))
    ab = kw.pop("abs_intervals", I.absorber_planes(nz, pml))
    return I.Problem(nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dz, theta_deg=theta, phi_deg=phi,
                     pml_planes=pml, z_ml=pml, abs_intervals=ab, cap=cap, pols=list(pols), **kw)


def oracle_setup(prob, a_bin):
    from oracle import psfd as O
    g = O.Grid(prob.to_dict(), prob.stack())
    fill = O.fill_fraction(a_bin, prob.zprofile(), prob.sigma_px)
    return g, fill


def rel_l2(a, b):
    a = torch.as_tensor(a).to(torch.complex128).cpu()
    b = torch.as_tensor(b).to(torch.complex128).cpu()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
