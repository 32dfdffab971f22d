"""GPU parity of the layered-background preconditioner (an addition to the paper's method).

The oracle builds each lateral mode's block of A0 (the operator with the contrast averaged over
every plane) by applying its full operator to unit sources and solves with LU in complex128.  The
GPU assembles the TE / TM blocks from closed forms and inverts them in FP32 with partial
pivoting, so this also checks the closed forms.  Tolerance: relative L2 1e-4 (the complex64 bar);
an FP32 inversion loses about cond(block) * 6e-8, and the blocks here stay below cond ~ 1e3.
"""
import numpy as np
import pytest
import torch

from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I
from tests.helpers import oracle_setup, problem, rel_l2

pytestmark = pytest.mark.gpu
TOL_C64 = 1e-4

GRIDS = [  # (nx, ny, nz, theta, phi, nrhs)
    (16, 16, 16, 6.0, 0.0, 1),
    (32, 16, 32, 8.0, 30.0, 2),
    (16, 32, 48, 4.0, 0.0, 1),
    (32, 32, 64, 6.0, 0.0, 2),
    (16, 16, 32, 0.0, 0.0, 4),
]


def setup(nx, ny, nz, theta, phi, nrhs, seed=1):
    from paper_2607_25330_b300 import psfd
    prob = problem(nx, ny, nz, theta=theta, phi=phi, pols=[i % 2 for i in range(nrhs)])
    a = I.mask_for(prob, seed, "manhattan")
    g, fill_o = oracle_setup(prob, a)
    plan = psfd.Plan(prob, nrhs=nrhs)
    fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    plan.layered_build()
    return prob, g, fill_o, plan, b


@pytest.mark.parametrize("grid", GRIDS)
def test_layered_precond_matches_oracle(grid):
    from paper_2607_25330_b300 import psfd
    prob, g, fill_o, plan, b = setup(*grid)
    # ky and -ky share their blocks when there is no Bloch shift along y (phi = 0)
    rows = grid[1] // 2 + 1 if grid[4] == 0.0 else grid[1]
    assert plan.layered_bytes() == grid[0] * rows * 5 * grid[2] ** 2 * 8
    x = torch.from_numpy(I.random_field(plan.shape, 3)).to(torch.complex64)
    y = plan.precond(x.cuda(), flags=psfd.PSFD_LAYERED).cpu()
    mats = O.layered_blocks(g, fill_o)
    for r in range(plan.nrhs):
        ref = O.apply_P_layered(g, fill_o, x[r].to(torch.complex128), mats)
        assert rel_l2(y[r], ref) < TOL_C64
    # the operator flag applies P, then A: the same as the two calls in sequence (A itself is
    # checked against the oracle by the operator tests).  The two routes differ by the complex64
    # rounding of P x and an extra pair of lateral transforms, which A amplifies by up to
    # max|k|^2 / k0^2 ~ 10 on these grids: 1e-4.
    z = plan.apply(x.cuda(), flags=psfd.PSFD_LAYERED).cpu()
    z2 = plan.apply(y.cuda()).cpu()
    assert rel_l2(z, z2) < 1e-4


def test_layered_is_the_inverse_for_a_laterally_uniform_fill():
    """With the same fill on every lateral point A0 = A: A P x = x up to the FP32 inversion."""
    from paper_2607_25330_b300 import psfd
    prob = problem(32, 32, 32, theta=6.0, pols=[0, 1])
    plan = psfd.Plan(prob, nrhs=2)
    fill = (torch.as_tensor(prob.zprofile(), dtype=torch.float32)[:, None, None] * 0.45).expand(32, 32, 32)
    fill = fill.contiguous().cuda()
    plan.background(prob.stack(), fill, prob.pols)
    plan.layered_build()
    x = torch.from_numpy(I.random_field(plan.shape, 5)).to(torch.complex64).cuda()
    y = plan.apply(x, flags=psfd.PSFD_LAYERED | psfd.PSFD_HYBRID)
    assert rel_l2(y.cpu(), x.cpu()) < 1e-4


def test_layered_solve_matches_oracle_and_converges_fast():
    from paper_2607_25330_b300 import psfd
    from oracle import krylov as K
    prob, g, fill_o, plan, b = setup(32, 32, 32, 6.0, 0.0, 2, seed=4)
    res = plan.solve_ex(b, tol=1e-6, maxit=400, method=psfd.PSFD_GMRES, restart=30, precond=psfd.PC_LAYERED)
    assert res["code"] == 0, res["info"]
    for r, inf in enumerate(res["info"]):
        assert inf["status"] == 0 and inf["r_rel"] <= 1e-6
        assert inf["iters"] <= 60, inf
        bo = O.source_b(g, fill_o, prob.pols[r])
        ref = K.solve(lambda E: O.apply_A(g, E, fill_o), lambda X: O.apply_M(g, X), bo, tol=1e-11,
                      maxit=4000, method="gmres", restart=60)
        assert ref["r_rel"] < 1e-10
        assert rel_l2(res["E"][r].cpu(), ref["E"]) < 1e-4


def test_layered_warm_start_refresh_and_state_errors():
    from paper_2607_25330_b300 import psfd
    prob = problem(16, 16, 16, theta=6.0, pols=[0])
    plan = psfd.Plan(prob, nrhs=1)
    x = torch.zeros(plan.shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(psfd.PsfdError):
        plan.layered_build()                       # no background yet
    fill = plan.mask_fill(torch.from_numpy(I.mask_for(prob, 2, "manhattan")), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    with pytest.raises(psfd.PsfdError):
        plan.solve_ex(b, tol=1e-6, maxit=10, precond=psfd.PC_LAYERED)   # blocks never built
    assert plan.layered_refresh(0.25)              # first call builds
    assert not plan.layered_refresh(0.25)          # same fill: nothing to do
    cold = plan.solve_ex(b, tol=1e-6, maxit=200, precond=psfd.PC_LAYERED)
    assert cold["code"] == 0
    # the exact solution as warm start needs no inner iteration
    warm = plan.solve_ex(b, x0=cold["E"].clone(), tol=1e-5, maxit=200, precond=psfd.PC_LAYERED)
    assert warm["info"][0]["iters"] == 0
    # another mask: the old blocks remain a valid preconditioner; refresh decides on the shift
    a2 = I.mask_for(prob, 9, "manhattan")
    fill2 = plan.mask_fill(torch.from_numpy(a2), prob.zprofile())
    b2 = plan.background(prob.stack(), fill2, prob.pols)
    stale = plan.solve_ex(b2, tol=1e-6, maxit=200, precond=psfd.PC_LAYERED)
    assert stale["code"] == 0
    shift = abs(float(np.mean(a2)) - float(np.mean(I.mask_for(prob, 2, "manhattan"))))
    assert plan.layered_refresh(0.0) == (shift > 0)
    fresh = plan.solve_ex(b2, tol=1e-6, maxit=200, precond=psfd.PC_LAYERED)
    assert fresh["code"] == 0
    assert rel_l2(fresh["E"].cpu(), stale["E"].cpu()) < 1e-4


def test_layered_full_size_128x128x64_reaches_1e6():
    """The 128x128x64, 2-rhs workload at 6 degrees: 1e-6 in the FP64 residual."""
    from paper_2607_25330_b300 import psfd
    prob = I.preset("manhattan_128x128x64")
    plan = psfd.Plan(prob)
    a = I.mask_for(prob, 11)
    fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    plan.layered_build()
    res = plan.solve_ex(b, tol=1e-6, maxit=600, method=psfd.PSFD_GMRES, restart=30, precond=psfd.PC_LAYERED,
                        out_c128=True)
    assert res["code"] == 0, res["info"]
    assert res["E"].dtype == torch.complex128
    g, fill_o = oracle_setup(prob, a)
    for r, inf in enumerate(res["info"]):
        assert inf["r_rel"] <= 1e-6 and inf["r_rel_output"] <= 1e-6 and inf["iters"] <= 200, inf
        # the returned FP64 field meets the tolerance in the oracle's own residual too
        bo = O.source_b(g, fill_o, prob.pols[r])
        assert O.rel_residual(g, res["E"][r].cpu(), fill_o, bo) <= 1.01e-6


@pytest.mark.parametrize("grid", [GRIDS[1], GRIDS[3]])
def test_half_storage_of_the_blocks(grid):
    """Blocks stored in half precision with a power-of-two scale per block: P x within the half
    rounding of its entries (2^-11 relative, amplified by cancellation in the sums: 2e-3) of the
    oracle's, half the bytes, and the same solve result."""
    from paper_2607_25330_b300 import psfd
    from oracle import krylov as K
    prob, g, fill_o, plan, b = setup(*grid)
    full = plan.layered_bytes()
    plan.layered_storage(True)
    plan.layered_build()
    assert plan.layered_bytes() * 2 == full
    x = torch.from_numpy(I.random_field(plan.shape, 3)).to(torch.complex64)
    y = plan.precond(x.cuda(), flags=psfd.PSFD_LAYERED).cpu()
    mats = O.layered_blocks(g, fill_o)
    for r in range(plan.nrhs):
        ref = O.apply_P_layered(g, fill_o, x[r].to(torch.complex128), mats)
        assert rel_l2(y[r], ref) < 2e-3
    res = plan.solve_ex(b, tol=1e-6, maxit=400, precond=psfd.PC_LAYERED, out_c128=True)
    assert res["code"] == 0
    bo = O.source_b(g, fill_o, prob.pols[0])
    assert O.rel_residual(g, res["E"][0].cpu(), fill_o, bo) <= 1.01e-6
    plan.layered_storage(False)
    with pytest.raises(psfd.PsfdError):
        plan.precond(x.cuda(), flags=psfd.PSFD_LAYERED)    # released until rebuilt


TC_GRIDS = [  # nz a multiple of 32: the half-precision blocks are applied on the tensor cores
    (32, 16, 32, 8.0, 30.0, 2),   # no ky / -ky pairing (Bloch shift along y)
    (32, 32, 64, 6.0, 0.0, 2),
    (16, 16, 32, 0.0, 0.0, 4),
    (16, 16, 64, 6.0, 0.0, 1),
    (32, 16, 32, 6.0, 0.0, 3),
    (16, 16, 64, 8.0, 30.0, 2),   # nz = 64 without pairing
]


@pytest.mark.parametrize("grid", TC_GRIDS)
def test_tensor_core_apply_of_half_blocks(grid, monkeypatch):
    """The tensor-core apply (f16 blocks, two-term f16 split of the vector, FP32 accumulation)
    against the SIMT apply of the same stored blocks (FP32 FMAs): the split keeps about 22 bits of
    the vector, so the two agree to a few FP32 roundings (1e-5), and P stays linear and
    scale-covariant to that level over 50 decades of input magnitude."""
    from paper_2607_25330_b300 import psfd
    prob, g, fill_o, plan, b = setup(*grid)
    plan.layered_storage(True)
    plan.layered_build()
    x1 = torch.from_numpy(I.random_field(plan.shape, 3)).to(torch.complex64).cuda()
    x2 = torch.from_numpy(I.random_field(plan.shape, 4)).to(torch.complex64).cuda()
    monkeypatch.setenv("PSFD_LAY_TC", "0")
    y_simt = plan.precond(x1, flags=psfd.PSFD_LAYERED).cpu()
    monkeypatch.setenv("PSFD_LAY_TC", "1")
    y1 = plan.precond(x1, flags=psfd.PSFD_LAYERED).cpu()
    for r in range(plan.nrhs):
        assert rel_l2(y1[r], y_simt[r]) < 1e-5
    y2 = plan.precond(x2, flags=psfd.PSFD_LAYERED).cpu()
    y12 = plan.precond(x1 + 3.0 * x2, flags=psfd.PSFD_LAYERED).cpu()
    assert rel_l2(y12, y1 + 3.0 * y2) < 1e-5
    for s in (1e-25, 1e25):
        ys = plan.precond(x1 * s, flags=psfd.PSFD_LAYERED).cpu()
        assert rel_l2(ys / s, y1) < 1e-5
    # a zero right-hand side stays zero (the scale of an all-zero column is finite)
    x0 = x1.clone()
    x0[0] = 0
    y0 = plan.precond(x0, flags=psfd.PSFD_LAYERED).cpu()
    assert torch.count_nonzero(y0[0]) == 0 and bool(torch.isfinite(torch.view_as_real(y0)).all())
    plan.device_status()


def test_tensor_core_apply_wait_gives_up_and_reports(monkeypatch):
    """The apply's wait for its bulk block copies is bounded: with no copy requested (a test hook;
    nothing else completes the barrier) every CTA gives up after about a second, records it, and
    leaves; psfd_device_status reports PSFD_ERR_TIMEOUT once, and the context stays usable."""
    from paper_2607_25330_b300 import psfd
    prob, g, fill_o, plan, b = setup(16, 16, 32, 0.0, 0.0, 2)
    plan.layered_storage(True)
    plan.layered_build()
    plan.device_status()
    monkeypatch.setenv("PSFD_LAY_TC", "1")
    x = torch.from_numpy(I.random_field(plan.shape, 3)).to(torch.complex64).cuda()
    y_ref = plan.precond(x, flags=psfd.PSFD_LAYERED).cpu()
    monkeypatch.setenv("PSFD_TEST_LAY_NO_COPY", "1")
    plan.precond(x, flags=psfd.PSFD_LAYERED)
    monkeypatch.delenv("PSFD_TEST_LAY_NO_COPY")
    with pytest.raises(psfd.PsfdError) as e:
        plan.device_status()
    assert e.value.code == psfd.PSFD_ERR_TIMEOUT and "layered" in str(e.value)
    plan.device_status()                                   # cleared
    y = plan.precond(x, flags=psfd.PSFD_LAYERED).cpu()     # and the next apply is complete again
    assert rel_l2(y, y_ref) == 0.0
    res = plan.solve_ex(b, tol=1e-6, maxit=400, precond=psfd.PC_LAYERED)
    assert res["code"] == 0


@pytest.mark.parametrize("half", [False, True])
def test_layered_solve_with_converged_right_hand_sides(half):
    """Right-hand sides that have converged are skipped by the layered apply and the operator kernels
    of every later iteration.  One rhs starts converged (its x0 is a solution), the other from zero:
    the active one must still reach the same field; with every rhs converged, nothing iterates and
    the field is x0 itself."""
    from paper_2607_25330_b300 import psfd
    prob = problem(64, 64, 64, theta=6.0, pols=[0, 1])
    a = I.mask_for(prob, 5, "manhattan")
    plan = psfd.Plan(prob, nrhs=2)
    fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    plan.layered_storage(half)
    plan.layered_build()
    ref = plan.solve_ex(b, tol=1e-9, maxit=400, method=psfd.PSFD_BICGSTAB, precond=psfd.PC_LAYERED,
                        inner_tol=1e-3, out_c128=True)
    assert all(i["status"] == 0 for i in ref["info"]), ref["info"]
    E_ref = ref["E"]
    # rhs 1 starts at (the complex64 rounding of) its solution: residual ~1e-6 < 1e-5
    x0 = torch.zeros(plan.shape, dtype=torch.complex64, device="cuda")
    x0[1] = E_ref[1].to(torch.complex64)
    res = plan.solve_ex(b, x0=x0, tol=1e-5, maxit=400, method=psfd.PSFD_BICGSTAB, precond=psfd.PC_LAYERED,
                        inner_tol=1e-3, out_c128=True)
    i0, i1 = res["info"]
    assert i0["status"] == 0 and i1["status"] == 0, res["info"]
    assert i1["iters"] == 0 and i0["iters"] > 0
    assert i0["r_rel"] <= 1e-5 and i1["r_rel"] <= 1e-5
    assert rel_l2(res["E"][1], x0[1]) < 1e-5     # x0 enters through a complex64 lateral transform
    assert rel_l2(res["E"][0], E_ref[0]) < 1e-3
    # every rhs converged from the start
    x0[0] = E_ref[0].to(torch.complex64)
    res2 = plan.solve_ex(b, x0=x0, tol=1e-5, maxit=400, method=psfd.PSFD_BICGSTAB, precond=psfd.PC_LAYERED,
                         inner_tol=1e-3, out_c128=True)
    assert all(i["status"] == 0 and i["iters"] == 0 for i in res2["info"]), res2["info"]
    assert rel_l2(res2["E"], x0) < 1e-5


@pytest.mark.parametrize("nz,half", [(32, False), (64, False), (64, True)])
def test_schur_form_equals_the_full_blocks(nz, half, monkeypatch):
    """The Schur form (TE^-1 and S^-1, E_z eliminated through the diagonal E_z-E_z block) and the
    full TE / TM inverses are two FP32 computations of the same exact inverse of A0."""
    from paper_2607_25330_b300 import psfd
    prob = problem(32, 32, nz, theta=6.0, pols=[0, 1])
    a = I.mask_for(prob, 7, "manhattan")
    x = torch.from_numpy(I.random_field((2, 3, nz, 32, 32), 8)).to(torch.complex64).cuda()
    out = {}
    for schur in ("0", "1"):
        monkeypatch.setenv("PSFD_LAY_SCHUR", schur)
        plan = psfd.Plan(prob, nrhs=2)
        plan.layered_storage(half)
        fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
        plan.background(prob.stack(), fill, prob.pols)
        plan.layered_build()
        # the Schur form keeps complex64 blocks even when half precision is requested
        per = (2 * nz * nz * 8) if schur == "1" else 5 * nz * nz * (4 if half else 8)
        assert plan.layered_bytes() == 32 * 17 * per
        out[schur] = plan.precond(x, flags=psfd.PSFD_LAYERED).cpu()
    e = rel_l2(out["1"], out["0"])
    print(f"Schur vs full blocks nz {nz} half {half}: rel L2 {e:.2e}")
    assert e < (2e-3 if half else 2e-4)


@pytest.mark.parametrize("grid", [(16, 16, 96, 6.0, 0.0, 2), (16, 16, 128, 4.0, 0.0, 1), (16, 16, 96, 6.0, 20.0, 1)])
def test_schur_layered_precond_matches_oracle(grid):
    """nz = 96 and 128 (the batched and fine-grid depths): P x against the oracle's LU of A0.

    Tolerance 1e-3: the Schur complement carries kappa^2 D Dg^-1 D, whose entries grow as
    1 / (kappa^2 - k0^2) for columns near grazing, so its FP32 inversion loses about three more
    digits than the full-block form's (measured 2.9e-4); P only steers the iteration, and the
    solves below reach the FP64 residual tolerance in a handful of iterations."""
    from paper_2607_25330_b300 import psfd
    prob, g, fill_o, plan, b = setup(*grid)
    assert plan.layered_bytes() == grid[0] * (grid[1] // 2 + 1 if grid[4] == 0.0 else grid[1]) * 2 * grid[2] ** 2 * 8
    x = torch.from_numpy(I.random_field(plan.shape, 3)).to(torch.complex64)
    y = plan.precond(x.cuda(), flags=psfd.PSFD_LAYERED).cpu()
    lu = torch.linalg.lu_factor(O.layered_blocks(g, fill_o))
    for r in range(plan.nrhs):
        ref = O.apply_P_layered(g, fill_o, x[r].to(torch.complex128), lu=lu)
        e = rel_l2(y[r], ref)
        print(f"Schur P {grid} rhs {r}: rel L2 {e:.2e}")
        assert e < 1e-3


@pytest.mark.parametrize("nz", [96, 128])
def test_schur_layered_solve_converges_fast(nz):
    """A 64x64 mask at nz = 96 / 128 with the Schur-form P: BiCGSTAB to 1e-6 (FP64 residual) in a few
    tens of iterations (measured 7; the paper's damping M with GMRES(30) has not reached 1e-8 after
    40000 iterations on the same masks), and the same field as GMRES(30) to 1e-10."""
    from paper_2607_25330_b300 import psfd
    prob = problem(64, 64, nz, theta=6.0, pols=[0, 1])
    a = I.mask_for(prob, 9, "manhattan")
    plan = psfd.Plan(prob, nrhs=2)
    fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
    b = plan.background(prob.stack(), fill, prob.pols)
    plan.layered_storage(True)
    plan.layered_build()
    res = plan.solve_ex(b, tol=1e-6, maxit=400, method=psfd.PSFD_BICGSTAB, precond=psfd.PC_LAYERED,
                        inner_tol=1e-3, out_c128=True)
    print(f"Schur P solve nz {nz}: {[(i['iters'], i['r_rel']) for i in res['info']]}")
    for i in res["info"]:
        assert i["status"] == 0 and i["r_rel"] <= 1e-6 and i["iters"] < 80, res["info"]
    # the residual above is the FP64 apply's (pinned to the oracle element-wise at 1e-14); the
    # field at 1e-6 lies within the operator's conditioning of the field at 1e-10
    ref = plan.solve_ex(b, tol=1e-10, maxit=400, method=psfd.PSFD_GMRES, restart=30, precond=psfd.PC_LAYERED,
                        inner_tol=1e-3, out_c128=True)
    assert all(i["status"] == 0 and i["r_rel"] <= 1e-10 for i in ref["info"]), ref["info"]
    assert rel_l2(res["E"], ref["E"]) < 1e-4


def test_layered_form_selects_the_schur_form_per_plan():
    """psfd_layered_form: the Schur form on request for nz a multiple of 32 (the same operator as the
    full blocks, two FP32 computations of one exact inverse), the full blocks at nz 48, and back to
    the default rule at the next build."""
    from paper_2607_25330_b300 import psfd
    cols = 32 * 17
    for nz in (64, 48):
        prob = problem(32, 32, nz, theta=6.0, pols=[0, 1])
        a = I.mask_for(prob, 7, "manhattan")
        x = torch.from_numpy(I.random_field((2, 3, nz, 32, 32), 8)).to(torch.complex64).cuda()
        plan = psfd.Plan(prob, nrhs=2)
        plan.layered_storage(True)
        fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
        plan.background(prob.stack(), fill, prob.pols)
        plan.layered_build()
        assert plan.layered_bytes() == cols * 5 * nz * nz * 4
        full = plan.precond(x, flags=psfd.PSFD_LAYERED).cpu()
        plan.layered_form(True)
        plan.layered_build()
        schur = nz % 32 == 0
        assert plan.layered_bytes() == cols * (2 * nz * nz * 8 if schur else 5 * nz * nz * 4)
        y = plan.precond(x, flags=psfd.PSFD_LAYERED).cpu()
        if schur:
            assert rel_l2(y, full) < 2e-3
        else:
            assert torch.equal(y, full)
        plan.layered_form(False)
        plan.layered_build()
        assert plan.layered_bytes() == cols * 5 * nz * nz * 4
        assert torch.equal(plan.precond(x, flags=psfd.PSFD_LAYERED).cpu(), full)
    assert psfd.lib().psfd_layered_form(None, 0) == psfd.PSFD_ERR_ARG
    assert psfd.lib().psfd_layered_form(plan.h, 7) == psfd.PSFD_ERR_ARG
