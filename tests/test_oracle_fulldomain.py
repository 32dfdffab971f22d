"""Pins of the full-domain PSFD mode (NEXT-3: the multilayer meshed in the domain, R = 0).

The bare Mo/Si multilayer, cell-averaged on the planes with an empty background stack, is solved
by the oracle's operator; the specular reflection of the scattered field above it must approach
the transfer-matrix reflection of the same stack (closed form) as the plane spacing shrinks.
"""
import math

import numpy as np
import pytest
import torch

from oracle import krylov as K
from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I
from tests.helpers import problem

PAIRS = 3


def bare_ml(nz, dz, theta, pol, nx=4):
    pml = int(round(4.0 / dz))    # 4 nm of PML at every spacing
    prob = problem(nx, nx, nz, theta=theta, pols=[pol], dx=150.0 / nx, dz=dz, pml_planes=pml, abs_intervals=1.0)
    g = O.Grid(prob.to_dict(), I.empty_stack())
    layers = []
    for _ in range(PAIRS):
        layers += [(I.N_SI ** 2, I.D_SI_NM), (I.N_MO ** 2, I.D_MO_NM)]
    z_top = (nz - pml - 6) * dz
    c = O.layered_cell_contrast(g, layers, z_top, I.N_SI ** 2)
    g.plane_contrast = c
    fill = torch.ones(nz, nx, nx, dtype=torch.float64)
    fill[c.abs() == 0] = 0.0
    stack = {"n": [n for _ in range(PAIRS) for n in (I.N_SI, I.N_MO)],
             "d": [d for _ in range(PAIRS) for d in (I.D_SI_NM, I.D_MO_NM)], "n_sub": I.N_SI}
    return prob, g, fill, z_top, stack


def solve_r(nz, dz, theta, pol):
    prob, g, fill, z_top, stack = bare_ml(nz, dz, theta, pol)
    b = O.source_b(g, fill, pol)
    res = K.solve(lambda E: O.apply_A(g, E, fill), None, b, tol=1e-11, maxit=3 * nz + 50, method="gmres",
                  restart=3 * nz + 20)
    assert res["r_rel"] < 1e-9
    r = O.specular_reflection(g, res["E"], int(round(z_top / dz)) + 3, z_top, pol)
    kpar2 = torch.tensor([[(g.k0 * math.sin(g.theta)) ** 2]], dtype=torch.float64)
    r_tmm = complex(O.reflection_coefficient(kpar2, stack, g.k0, "s" if pol == 0 else "p")[0, 0])
    return r, r_tmm


@pytest.mark.parametrize("theta,pol", [(0.0, 0), (10.37, 0), (10.37, 1)])
def test_meshed_multilayer_reflection_converges_to_transfer_matrix(theta, pol):
    r1, t1 = solve_r(64, 0.5, theta, pol)
    r2, t2 = solve_r(128, 0.25, theta, pol)
    e1, e2 = abs(r1 - t1), abs(r2 - t2)
    assert abs(t1 - t2) < 1e-12
    # cell-averaged interfaces: second order in dz (measured ratios 3.6-4.2 for a halving)
    assert e2 < 0.35 * e1, (e1, e2)
    assert e2 < 0.005 * abs(t2), (r2, t2)


def test_plane_contrast_table_reproduces_the_absorber_default():
    prob = problem(4, 4, 16, theta=6.0, pols=[0])
    g = O.Grid(prob.to_dict(), prob.stack())
    a = I.mask_for(prob, 3, "manhattan")
    fill = O.fill_fraction(a, prob.zprofile(), 1.0)
    x = torch.from_numpy(I.random_field(g.shape, 2))
    y0 = O.apply_A(g, x, fill)
    g.plane_contrast = torch.full((16,), g.deps_abs, dtype=torch.complex128)
    y1 = O.apply_A(g, x, fill)
    assert torch.equal(y0, y1)
