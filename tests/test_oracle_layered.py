"""Pins of the oracle's layered-background preconditioner (an addition to the paper's method).

P = A0^-1 where A0 is the operator of Eqs. bg_source / vector_helmholtz_operator with the contrast
replaced on every plane by its lateral mean.  Facts fixed outside the oracle's own construction:
* a laterally uniform fill makes A0 = A, so P is the exact inverse of the full operator
  (checked through apply_A, the same operator the slab and dense-LU pins fix);
* in a laterally uniform medium TE and TM decouple: in the (s, t, z) basis of each lateral
  mode the blocks coupling E_s with (E_t, E_z) vanish (Maxwell's equations in layered media);
* the blocks are the modes' restrictions of A0: A0 x computed by the full operator with the mean
  fill equals the per-mode matrices applied to the lateral DFT of x.
"""
import numpy as np
import torch

from oracle import krylov as K
from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I
from tests.helpers import problem

C128 = torch.complex128


def _setup(nx=8, ny=8, nz=16, theta=6.0, uniform=False, seed=3):
    prob = problem(nx, ny, nz, theta=theta, pols=[0])
    g = O.Grid(prob.to_dict(), prob.stack())
    if uniform:
        fill = torch.as_tensor(prob.zprofile(), dtype=torch.float64)[:, None, None].expand(nz, ny, nx) * 0.45
        fill = fill.contiguous()
    else:
        a = I.manhattan_mask(ny, nx, np.random.default_rng(seed), nrect=(2, 4), edge=(2, 5))
        fill = O.fill_fraction(a, prob.zprofile(), 1.0)
    return prob, g, fill


def test_uniform_fill_makes_P_the_exact_inverse_of_A():
    prob, g, fill = _setup(uniform=True)
    x = torch.from_numpy(I.random_field(g.shape, 7))
    y = O.apply_P_layered(g, fill, O.apply_A(g, x, fill))
    assert float(torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)) < 1e-10
    # and the other order
    z = O.apply_A(g, O.apply_P_layered(g, fill, x), fill)
    assert float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)) < 1e-10
    # the same blocks factored once (LU with partial pivoting) and applied by triangular solves
    lu = torch.linalg.lu_factor(O.layered_blocks(g, fill))
    w = O.apply_P_layered(g, fill, O.apply_A(g, x, fill), lu=lu)
    assert float(torch.linalg.vector_norm(w - x) / torch.linalg.vector_norm(x)) < 1e-10


def test_blocks_decouple_te_from_tm():
    prob, g, fill = _setup()
    mats = O.layered_blocks(g, fill)
    nz = g.nz
    for iy in range(g.ny):
        for ix in range(g.nx):
            sx, sy, tx, ty = (complex(v[iy, ix]) for v in (g.sx, g.sy, g.tx, g.ty))
            # rotation (x, y, z) -> (s, t, z) on every plane
            Rm = torch.zeros(3 * nz, 3 * nz, dtype=C128)
            eye = torch.eye(nz, dtype=C128)
            Rm[:nz, :nz], Rm[:nz, nz:2 * nz] = sx * eye, sy * eye
            Rm[nz:2 * nz, :nz], Rm[nz:2 * nz, nz:2 * nz] = tx * eye, ty * eye
            Rm[2 * nz:, 2 * nz:] = eye
            B = Rm @ mats[iy, ix] @ Rm.T          # Rm is real orthogonal
            scale = float(B.abs().max())
            assert float(B[:nz, nz:].abs().max()) < 1e-12 * scale
            assert float(B[nz:, :nz].abs().max()) < 1e-12 * scale


def test_blocks_reproduce_the_mean_fill_operator():
    prob, g, fill = _setup(nx=8, ny=4, nz=16, seed=5)
    mats = O.layered_blocks(g, fill)
    x = torch.from_numpy(I.random_field(g.shape, 9))
    ref = O.apply_A(g, x, O.lateral_mean_fill(fill))
    xh = torch.fft.fft2(x, dim=(-2, -1)).permute(2, 3, 0, 1).reshape(g.ny, g.nx, 3 * g.nz, 1)
    yh = (mats @ xh).reshape(g.ny, g.nx, 3, g.nz).permute(2, 3, 0, 1)
    y = torch.fft.ifft2(yh, dim=(-2, -1))
    assert float(torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)) < 1e-12


def test_preconditioned_solve_reaches_the_dense_solution():
    """GMRES on A P y = b, E = P y, gives the solution of A E = b (dense LU on a tiny grid)."""
    prob, g, fill = _setup(nx=4, ny=4, nz=8, seed=11)
    b = O.source_b(g, fill, 0)
    mats = O.layered_blocks(g, fill)
    P = lambda X: O.apply_P_layered(g, fill, X, mats)
    res = K.solve(lambda E: O.apply_A(g, E, fill), P, b, tol=1e-12, maxit=300, method="gmres", restart=40)
    ref = K.dense_solve(K.dense_matrix(lambda E: O.apply_A(g, E, fill), g.shape), b)
    assert float(torch.linalg.vector_norm(res["E"] - ref) / torch.linalg.vector_norm(ref)) < 1e-9
