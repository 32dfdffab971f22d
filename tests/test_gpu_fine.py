"""The fine-discretisation workload at full size: 512x512x128 (0.5 nm lateral pixels), TE + TM at
6 deg, warm start from a 128x128x32 FNO prediction upsampled spectrally, GMRES(30).

At this size (1e8 unknowns per polarisation) the checks are properties that hold at any size:
the plane-wave symbol of the operator (Eq. vector_helmholtz_operator), the adjoint identity,
exact interpolation of the spectral upsampling at the coarse grid points, and a bounded
warm-started solve whose FP64 residual decreases monotonically.
"""
import numpy as np
import pytest
import torch

from paper_2607_25330_b300 import inputs as I
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fine():
    from paper_2607_25330_b300 import psfd
    prob = I.preset("fine_512x512x128")
    a = I.mask_for(prob, 5, "manhattan_dense")
    plan = psfd.Plan(prob)
    fill = plan.mask_fill(torch.from_numpy(a).cuda(), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    return prob, plan, fill, b


def test_plane_wave_symbol_at_full_size():
    """No PML, no contrast: a grid plane wave is an eigenfunction with the closed-form symbol."""
    from paper_2607_25330_b300 import psfd
    prob = I.preset("fine_512x512x128")
    prob.pml_planes = 0
    plan = psfd.Plan(prob, nrhs=1)
    fill = torch.zeros((prob.nz, prob.ny, prob.nx), dtype=torch.float32, device="cuda")
    plan.background(prob.stack(), fill, [0])
    k0 = 2 * np.pi / prob.lam
    kxi = k0 * np.sin(np.radians(prob.theta_deg))
    mx, my, mz = 37, -101, 19
    kk = np.array([2 * np.pi * mx / (prob.nx * prob.dx), 2 * np.pi * my / (prob.ny * prob.dy),
                   2 * np.pi * mz / (prob.nz * prob.dz)])
    k = kk + np.array([kxi, 0.0, 0.0])
    x = torch.arange(prob.nx, dtype=torch.float64, device="cuda") * prob.dx
    y = torch.arange(prob.ny, dtype=torch.float64, device="cuda") * prob.dy
    z = torch.arange(prob.nz, dtype=torch.float64, device="cuda") * prob.dz
    ph = torch.exp(1j * (kk[2] * z[:, None, None] + kk[1] * y[None, :, None] + kk[0] * x[None, None, :]))
    e = np.array([0.3 + 0.2j, -0.5 + 0.1j, 0.25 - 0.4j])
    E = torch.stack([complex(c) * ph for c in e])[None].to(torch.complex64).contiguous()
    out = plan.apply(E)
    sym = (k @ k) * e - k * (k @ e) - k0 ** 2 * e
    ref = torch.stack([complex(c) * ph for c in sym])[None]
    assert rel_l2(out.cpu(), ref.cpu()) < 1e-4


def test_adjoint_identity_at_full_size(fine):
    from paper_2607_25330_b300 import psfd
    prob, plan, fill, b = fine
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(plan.shape, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.randn(plan.shape, dtype=torch.complex64, device="cuda", generator=g)
    for f in (0, psfd.PSFD_PRECOND):
        Ax = plan.apply(x, flags=f)
        AHy = plan.apply(y, flags=f | psfd.PSFD_ADJOINT)
        lhs = torch.vdot(Ax.flatten().to(torch.complex128), y.flatten().to(torch.complex128))
        rhs = torch.vdot(x.flatten().to(torch.complex128), AHy.flatten().to(torch.complex128))
        assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))
        del Ax, AHy


def test_warm_start_from_upsampled_coarse_fno(fine):
    from paper_2607_25330_b300 import psfd
    prob, plan, fill, b = fine
    coarse = I.preset("fno_coarse_128x128x32")
    S = I.FNOShape()
    models = []
    for pol in prob.pols:
        w = I.fno_weights(S, 77 + pol)
        models.append(psfd.fno_struct({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in w.items()}, S))
    # coarse input: the same layout on the coarse grid (every 4th pixel), smoothed on that grid
    a_fine = I.mask_for(prob, 5, "manhattan_dense")
    cplan = psfd.Plan(coarse, nrhs=1)
    cfill = cplan.mask_fill(torch.from_numpy(np.ascontiguousarray(a_fine[::4, ::4])).cuda(), coarse.zprofile())
    Ec = torch.cat([psfd.fno_forward(m, cfill[None].contiguous()) for m in models])   # (2, 3, 32, 128, 128)
    x0 = psfd.spectral_upsample(Ec, prob.nz, prob.ny, prob.nx)                       # (2, 3, 128, 512, 512)
    # zero-padded spectral interpolation passes exactly through the coarse samples
    assert rel_l2(x0[:, :, ::4, ::4, ::4].cpu(), Ec.cpu()) < 1e-5
    res = plan.solve_ex(b, x0=x0.contiguous(), tol=1e-6, maxit=60, method=psfd.PSFD_GMRES, restart=30,
                        inner_tol=1e-2, max_outer=2)
    for r in range(2):
        info = res["info"][r]
        assert info["iters"] > 0 and np.isfinite(info["r_rel"])
        assert info["r_rel"] < info["r_rel_initial"]


def test_fine_grid_reaches_1e6_with_layered_schur_P(fine):
    """The fine-discretisation workload to its tolerance: 512x512x128, TE + TM at 6 deg, GMRES(30)
    in FP64 refinement with the layered P in the Schur form (nz = 128, complex64 blocks, 34 GB),
    cold and warm from the upsampled 128x128x32 prediction; FP64 residual of the returned FP64
    field <= 1e-6 (its operator is the FP64 apply pinned element-wise to the oracle)."""
    from paper_2607_25330_b300 import psfd
    prob, plan, fill, b = fine
    plan.layered_build()
    assert plan.layered_bytes() == 512 * 257 * 2 * 128 * 128 * 8
    cold = plan.solve_ex(b, tol=1e-6, maxit=400, method=psfd.PSFD_GMRES, restart=30, precond=psfd.PC_LAYERED,
                         inner_tol=1e-3, out_c128=True)
    print("fine grid cold:", [(i["iters"], i["r_rel"]) for i in cold["info"]])
    for i in cold["info"]:
        assert i["status"] == 0 and i["r_rel"] <= 1e-6 and i["iters"] < 100, cold["info"]
    coarse = I.preset("fno_coarse_128x128x32")
    S = I.FNOShape()
    cplan = psfd.Plan(coarse, nrhs=1)
    a_fine = I.mask_for(prob, 5, "manhattan_dense")
    cfill = cplan.mask_fill(torch.from_numpy(np.ascontiguousarray(a_fine[::4, ::4])).cuda(), coarse.zprofile())
    Ec = torch.cat([psfd.fno_forward(psfd.fno_struct({k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
                                                      for k, v in I.fno_weights(S, 77 + pol).items()}, S),
                                     cfill[None].contiguous()) for pol in prob.pols])
    x0 = psfd.spectral_upsample(Ec, prob.nz, prob.ny, prob.nx).contiguous()
    warm = plan.solve_ex(b, x0=x0, tol=1e-6, maxit=400, method=psfd.PSFD_GMRES, restart=30,
                         precond=psfd.PC_LAYERED, inner_tol=1e-3, out_c128=True)
    print("fine grid warm:", [(i["iters"], i["r_rel"], i["r_rel_initial"]) for i in warm["info"]])
    for i in warm["info"]:
        assert i["status"] == 0 and i["r_rel"] <= 1e-6, warm["info"]
    assert rel_l2(warm["E"], cold["E"]) < 1e-4
