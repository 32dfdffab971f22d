"""Pins of the oracle's Krylov solves: dense LU on tiny grids and the warm-start identities.

Eqs. right_preconditioned, right_correction_solution, right_preconditioned_system,
relative_residual (Sec. 3, PINO warm start for preconditioned PSFD).
"""
import numpy as np
import pytest
import torch

from oracle import krylov as K
from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I


def tiny(theta=6.0, **kw):
    p = I.Problem(nx=4, ny=4, nz=8, dx=2.0, dy=2.0, dz=2.0, theta_deg=theta, pml_planes=2, z_ml=2,
                  abs_intervals=3.0, cap=True, **kw)
    g = O.Grid(p.to_dict(), I.multilayer_stack(True))
    a = I.manhattan_mask(4, 4, np.random.default_rng(3), nrect=(2, 3), edge=(1, 2))
    fill = O.fill_fraction(a, p.zprofile(), 1.0)
    return p, g, fill


@pytest.fixture(scope="module")
def system():
    p, g, fill = tiny()
    A = lambda E: O.apply_A(g, E, fill)
    Amat = K.dense_matrix(A, g.shape)
    b = O.source_b(g, fill, 0)
    x_lu = K.dense_solve(Amat, b)
    return p, g, fill, A, b, x_lu


@pytest.mark.parametrize("method", ["bicgstab", "gmres"])
@pytest.mark.parametrize("precond", [False, True])
def test_krylov_matches_dense_lu(system, method, precond):
    """The Krylov solution equals the LU solution of the assembled operator (384 unknowns)."""
    p, g, fill, A, b, x_lu = system
    M = (lambda x: O.apply_M(g, x)) if precond else None
    res = K.solve(A, M, b, tol=1e-13, maxit=3000, method=method, restart=30)
    assert res["status"] == 0
    assert res["r_rel"] < 1e-12
    err = float(torch.linalg.vector_norm(res["E"] - x_lu) / torch.linalg.vector_norm(x_lu))
    assert err < 1e-9


def test_operator_is_nonsingular_and_moderately_conditioned(system):
    p, g, fill, A, b, x_lu = system
    Amat = K.dense_matrix(A, g.shape)
    s = torch.linalg.svdvals(Amat)
    kappa = float(s[0] / s[-1])
    assert np.isfinite(kappa) and kappa < 1e6


def test_warm_start_from_the_exact_solution_needs_no_iterations(system):
    """E_base = solution: b - A E_base ~ 0, so y = 0 and E = E_base (Eq. right_correction_solution)."""
    p, g, fill, A, b, x_lu = system
    res = K.solve(A, lambda x: O.apply_M(g, x), b, E_base=x_lu, tol=1e-8)
    assert res["iters"] == 0
    assert float((res["E"] - x_lu).abs().max()) == 0.0


def test_zero_warm_start_is_the_cold_solve(system):
    """E_base = 0 reduces the affine system to A M x = b (Eq. right_preconditioned)."""
    p, g, fill, A, b, x_lu = system
    M = lambda x: O.apply_M(g, x)
    h1, h2 = [], []
    r1 = K.solve(A, M, b, E_base=None, tol=1e-8, history=h1)
    r2 = K.solve(A, M, b, E_base=torch.zeros_like(b), tol=1e-8, history=h2)
    assert r1["iters"] == r2["iters"]
    assert np.allclose(h1, h2, rtol=1e-12, atol=0)
    assert float((r1["E"] - r2["E"]).abs().max()) < 1e-14 * float(r1["E"].abs().max())


def test_relative_residual_uses_the_original_rhs(system):
    """Eq. relative_residual normalises by ||b||, also when warm-started (not by ||b - A E_base||)."""
    p, g, fill, A, b, x_lu = system
    E0 = 0.9 * x_lu
    res = K.solve(A, lambda x: O.apply_M(g, x), b, E_base=E0, tol=1e-6)
    true = float(torch.linalg.vector_norm(b - A(res["E"])) / torch.linalg.vector_norm(b))
    assert abs(res["r_rel"] - true) < 1e-15
    assert true <= 1.5e-6
    # the warm start lowers the number of iterations against the cold solve
    cold = K.solve(A, lambda x: O.apply_M(g, x), b, tol=1e-6)
    assert res["iters"] <= cold["iters"]
