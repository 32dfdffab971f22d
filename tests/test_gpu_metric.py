"""GPU parity of the threshold-contour width metric (Sec. 4, Eq. logistic_sigmoid) against the
oracle on the same complex64 fields.  Segment counts (float32 above/below decisions on both sides)
are compared exactly; widths and deviations to 1e-4 pixel (float32 crossing interpolation)."""
import numpy as np
import pytest
import torch

from oracle import metric as MT
from paper_2607_25330_b300 import inputs as I
from tests.helpers import problem

pytestmark = pytest.mark.gpu


def _top_plane(prob):
    zp = np.asarray(prob.zprofile())
    return int(np.nonzero(zp > 0)[0].max()) + 1


def _check(plan, E, Eref, z, I_th, dx):
    g = plan.width_metric(E, Eref, z, I_th=I_th)
    o = MT.deviation(E[0].cpu().numpy(), Eref[0].cpu().numpy(), z, I_th=I_th, n_lines=100, dx=dx, dy=dx)
    assert g["matched"] == o["matched"] and g["unresolved"] == o["unresolved"]
    assert abs(g["mean"] - o["mean"]) <= 1e-4 * dx / 4 + 1e-6 * abs(o["mean"])
    assert abs(g["max"] - o["max"]) <= 1e-4 * dx / 4 + 1e-6 * abs(o["max"])
    return g


def test_width_metric_of_partial_solves_matches_oracle():
    from paper_2607_25330_b300 import psfd
    prob = problem(64, 64, 32, theta=6.0, pols=[0])
    plan = psfd.Plan(prob, nrhs=1)
    fill = plan.mask_fill(torch.from_numpy(I.mask_for(prob, 7, "manhattan")), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    plan.layered_build()
    ref = plan.solve_ex(b, tol=1e-7, maxit=400, precond=psfd.PC_LAYERED)["E"].clone()
    z = _top_plane(prob)
    Iref = (ref[0, 1, z].abs() ** 2).cpu().numpy()
    seen = 0
    for k in (1, 2, 4):
        E = plan.solve(b, tol=1e-12, maxit=k, method=psfd.PSFD_GMRES, restart=30, precond=psfd.PC_LAYERED)["E"]
        for I_th in (0.15, float(np.median(Iref))):
            g = _check(plan, E, ref, z, I_th, prob.dx)
            seen += g["matched"] + g["unresolved"]
    assert seen > 0
    # the converged field against itself: no deviation
    g = _check(plan, ref, ref, z, float(np.median(Iref)), prob.dx)
    assert g["mean"] == 0.0 and g["unresolved"] == 0 and g["matched"] > 0


def test_width_metric_closed_form_on_a_triangle_wave():
    """Intensity linear between samples: every row segment narrows by exactly 3.2 px."""
    from paper_2607_25330_b300 import psfd
    prob = problem(64, 16, 16, theta=0.0, pols=[0])
    plan = psfd.Plan(prob, nrhs=1)

    def field(level):
        x = np.arange(64)
        ph = (x % 32) / 32
        tri = 1.0 - 4.0 * np.minimum(ph, 1.0 - ph)
        Irow = (0.15 + 0.1 * (tri - level)).astype(np.float32)
        E = torch.zeros(plan.shape, dtype=torch.complex64)
        E[0, 1, 3] = torch.from_numpy(np.sqrt(np.maximum(Irow, 0))).float()[None, :].expand(16, 64)
        return E.cuda()

    g = plan.width_metric(field(0.5), field(0.3), 3, I_th=0.15)
    assert g["matched"] == 2 * 16 and g["unresolved"] == 0
    assert abs(g["mean"] - 3.2 * 2.0 / 4.0) < 1e-4 and g["frac_above_1nm"] == 1.0
