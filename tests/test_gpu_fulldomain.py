"""Full-domain PSFD on the GPU (NEXT-3): the bare Mo/Si multilayer meshed in the domain (per-plane
contrast from psfd_set_layer_stack_contrast, empty background stack so R = 0), lit at the
representable angles of a 150 nm period (Sec. 3: 0, 5.16, 10.37, 15.66 deg), TE and TM.

The specular reflection of the GPU field is compared with the oracle's solution of the same
discretisation (FP64 fields on both sides: 1e-6) and with the transfer-matrix reflection of the
stack (cell-averaged interfaces: 1.2 % at 0.5 nm planes, 0.4 % at 0.25 nm, second order)."""
import math

import numpy as np
import pytest
import torch

from oracle import krylov as K
from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I
from tests.helpers import problem

pytestmark = pytest.mark.gpu
PAIRS = 3


def stack():
    return {"n": [n for _ in range(PAIRS) for n in (I.N_SI, I.N_MO)],
            "d": [d for _ in range(PAIRS) for d in (I.D_SI_NM, I.D_MO_NM)], "n_sub": I.N_SI}


def run(theta, nz, dz, precond, restart):
    from paper_2607_25330_b300 import psfd
    pml = int(round(4.0 / dz))
    prob = problem(16, 16, nz, theta=theta, pols=[0, 1], dx=150.0 / 16, dz=dz, pml_planes=pml, abs_intervals=1.0)
    z_top = (nz - pml - 6) * dz
    plan = psfd.Plan(prob, nrhs=2)
    zm = plan.set_layer_stack_contrast(stack(), z_top)
    fill = plan.mask_fill(torch.ones(16, 16, dtype=torch.uint8), zm)
    b = plan.background(I.empty_stack(), fill, [0, 1])
    if precond == psfd.PC_LAYERED:
        plan.layered_build()
    res = plan.solve_ex(b, tol=1e-9, maxit=3000, precond=precond, restart=restart, out_c128=True)
    assert res["code"] == 0, res["info"]
    g = O.Grid(prob.to_dict(), I.empty_stack())
    layers = [(n * n, d) for n, d in zip(stack()["n"], stack()["d"])]
    g.plane_contrast = O.layered_cell_contrast(g, layers, z_top, I.N_SI ** 2)
    fill_o = torch.from_numpy(np.repeat(zm[:, None, None], 16, 1).repeat(16, 2)).double()
    z_obs = int(round(z_top / dz)) + 3
    kpar2 = torch.tensor([[(g.k0 * math.sin(g.theta)) ** 2]], dtype=torch.float64)
    out = []
    for r, pol in enumerate((0, 1)):
        E = res["E"][r].cpu()
        r_gpu = O.specular_reflection(g, E, z_obs, z_top, pol)
        bo = O.source_b(g, fill_o, pol)
        ref = K.solve(lambda X: O.apply_A(g, X, fill_o), None, bo, tol=1e-11, maxit=3 * nz + 60,
                      method="gmres", restart=3 * nz + 30)
        r_or = O.specular_reflection(g, ref["E"], z_obs, z_top, pol)
        r_tmm = complex(O.reflection_coefficient(kpar2, stack(), g.k0, "s" if pol == 0 else "p")[0, 0])
        out.append((r_gpu, r_or, r_tmm))
    return out


@pytest.mark.parametrize("theta", [0.0, 5.16, 10.37, 15.66])
def test_bare_multilayer_reflection_at_representable_angles(theta):
    from paper_2607_25330_b300 import psfd
    for r_gpu, r_or, r_tmm in run(theta, 64, 0.5, psfd.PC_LAYERED, 30):
        assert abs(r_gpu - r_or) < 1e-6 * max(1.0, abs(r_or)), (r_gpu, r_or)
        assert abs(r_gpu - r_tmm) < 0.012 * abs(r_tmm), (r_gpu, r_tmm)


def test_bare_multilayer_refinement_converges_at_second_order():
    """0.25 nm planes (nz = 128, no layered blocks at this depth: spectral damping M, GMRES(256))."""
    from paper_2607_25330_b300 import psfd
    coarse = run(10.37, 64, 0.5, psfd.PC_LAYERED, 30)
    fine = run(10.37, 128, 0.25, psfd.PC_DAMPING, 256)
    for (rc, _, tc), (rf, of, tf) in zip(coarse, fine):
        assert abs(rf - of) < 1e-6 * max(1.0, abs(of))
        assert abs(rf - tf) < 0.35 * abs(rc - tc) and abs(rf - tf) < 0.005 * abs(tf)
