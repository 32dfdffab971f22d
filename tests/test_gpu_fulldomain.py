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
from tests.helpers import problem, rel_l2

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
    zo = (g.plane_contrast.abs() > 0).double()                 # the oracle's own plane mask
    assert np.array_equal(zo.numpy(), zm.astype(np.float64))
    fill_o = zo[:, None, None].expand(nz, 16, 16).contiguous()
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


def _ml40_run(nz, dz, theta):
    """The whole 40-pair Mo/Si stack (280 nm, Si substrate) meshed on nz planes of dz (Fig. 1(c,d)
    setting), 16 x 16 lateral, TE + TM; GMRES(256) with the damping M in FP64 refinement to 1e-8."""
    from paper_2607_25330_b300 import psfd
    st = I.multilayer_stack(False)
    pml = int(round(4.0 / dz))
    prob = problem(16, 16, nz, theta=theta, pols=[0, 1], dx=150.0 / 16, dz=dz, pml_planes=pml, abs_intervals=1.0,
                   cap=False)
    z_top = (nz - pml - 6) * dz
    plan = psfd.Plan(prob, nrhs=2)
    zm = plan.set_layer_stack_contrast(st, z_top)
    assert zm.sum() >= 280.0 / dz                    # every stack plane carries contrast
    fill = plan.mask_fill(torch.ones(16, 16, dtype=torch.uint8), zm)
    b = plan.background(I.empty_stack(), fill, [0, 1])
    res = plan.solve_ex(b, tol=1e-8, maxit=20000, method=psfd.PSFD_GMRES, restart=256, precond=psfd.PC_DAMPING,
                        inner_tol=1e-2, out_c128=True)
    assert res["code"] == 0, res["info"]
    g = O.Grid(prob.to_dict(), I.empty_stack())
    kpar2 = torch.tensor([[(g.k0 * math.sin(g.theta)) ** 2]], dtype=torch.float64)
    z_obs = int(round(z_top / dz)) + 3
    out = []
    for r, pol in enumerate((0, 1)):
        r_gpu = O.specular_reflection(g, res["E"][r].cpu(), z_obs, z_top, pol)
        r_tmm = complex(O.reflection_coefficient(kpar2, st, g.k0, "s" if pol == 0 else "p")[0, 0])
        out.append((r_gpu, r_tmm))
    return out


@pytest.mark.parametrize("theta", [0.0, 5.16, 10.37, 15.66])
def test_full_40_pair_multilayer_converges_to_transfer_matrix(theta):
    """NEXT-3 at the paper's scale: the bare 40-pair multilayer meshed at 1 nm (nz = 512) and 0.5 nm
    (nz = 1024) planes; the specular reflection of the full-domain solve approaches the
    transfer-matrix reflection as the planes halve.  Measured |r_gpu - r_tmm| / |r_tmm|:
    1.7 % -> 0.51 % at 0 deg, 1.1 % -> 0.36 % at 5.16, 4.1 % -> 0.25 % at 10.37 (|r| ~ 0.85, in the
    Bragg band) and 17 % -> 3.2 % at 15.66 deg (|r| = 0.28, off the band); the absolute error at
    0.5 nm is below 0.009 at every angle."""
    coarse = _ml40_run(512, 1.0, theta)
    fine = _ml40_run(1024, 0.5, theta)
    for (rc, tc), (rf, tf) in zip(coarse, fine):
        ec, ef = abs(rc - tc) / abs(tc), abs(rf - tf) / abs(tf)
        print(f"40 pairs, {theta} deg: |r_tmm| {abs(tf):.4f}; error 1 nm {ec:.2e}, 0.5 nm {ef:.2e}")
        assert abs(tc - tf) < 1e-12
        assert abs(rf - tf) < 0.01 and ef < 0.5 * ec


@pytest.mark.parametrize("nz,dz", [(256, 1.0), (512, 1.0), (1024, 0.5)])
def test_long_column_operator_matches_oracle(nz, dz):
    """The axial kernels at 256, 512 and 1024 planes (one warp per column): A, A M and A^H of a
    meshed stack against the oracle, complex64 and FP64 applies."""
    from paper_2607_25330_b300 import psfd
    st = I.multilayer_stack(False)
    pml = int(round(4.0 / dz))
    prob = problem(16, 16, nz, theta=6.0, pols=[0], dx=150.0 / 16, dz=dz, pml_planes=pml, abs_intervals=1.0, cap=False)
    z_top = (nz - pml - 6) * dz
    plan = psfd.Plan(prob, nrhs=1)
    zm = plan.set_layer_stack_contrast(st, z_top)
    g = O.Grid(prob.to_dict(), I.empty_stack())
    layers = [(n * n, d) for n, d in zip(st["n"], st["d"])]
    g.plane_contrast = O.layered_cell_contrast(g, layers, z_top, st["n_sub"] ** 2)
    zo = (g.plane_contrast.abs() > 0).double()
    assert np.array_equal(zo.numpy(), zm.astype(np.float64))
    # a patterned binary fill on every stack plane, given to both sides directly (exact in float32)
    rng = np.random.default_rng(4)
    a = torch.from_numpy((rng.random((16, 16)) > 0.3).astype(np.float64))
    fill_o = zo[:, None, None] * a[None]
    plan.background(I.empty_stack(), fill_o.float().cuda(), [0])
    x = torch.from_numpy(I.random_field(plan.shape, 5))
    for flags in (0, psfd.PSFD_PRECOND, psfd.PSFD_ADJOINT):
        y = plan.apply(x.to(torch.complex64).cuda(), flags=flags).cpu()
        xr = x[0]
        if flags == psfd.PSFD_ADJOINT:
            ref = O.apply_AH(g, xr, fill_o)
        else:
            ref = O.apply_A(g, O.apply_M(g, xr) if flags else xr, fill_o)
        e = rel_l2(y[0], ref)
        print(f"nz {nz} flags {flags}: rel L2 {e:.2e}")
        assert e < 1e-4
    y64 = plan.apply64(x.cuda()).cpu()
    e64 = rel_l2(y64[0], O.apply_A(g, x[0], fill_o))
    print(f"nz {nz} FP64 apply: rel L2 {e64:.2e}")
    assert e64 < 1e-10
