"""Batched multi-mask solve (masks of uneven lateral size and depth, several angles and both
polarisations) and the FFT tile autotuner."""
import numpy as np
import pytest
import torch

from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I
from tests.helpers import oracle_setup, problem, rel_l2

pytestmark = pytest.mark.gpu


def make(nx, nz, theta, seed):
    from paper_2607_25330_b300 import psfd
    prob = problem(nx, nx, nz, theta=theta, pols=[0, 1])
    a = I.mask_for(prob, seed)
    plan = psfd.Plan(prob, stream=torch.cuda.Stream())
    with torch.cuda.stream(plan.stream):
        fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
        b = plan.background(prob.stack(), fill, prob.pols)
    plan.stream.synchronize()
    return prob, a, plan, fill, b


def test_batched_solve_equals_individual_solves():
    from paper_2607_25330_b300 import psfd
    specs = [(32, 32, 4.0, 1), (64, 48, 6.0, 2), (96, 32, 8.0, 3), (64, 64, 4.0, 4), (32, 48, 8.0, 5), (128, 32, 6.0, 6)]
    items = [make(*s) for s in specs]
    plans = [it[2] for it in items]
    bs = [it[4] for it in items]
    Es, infos = psfd.solve_batched(plans, bs, tol=1e-3, maxit=3000, method=psfd.PSFD_GMRES, restart=30)
    torch.cuda.synchronize()
    for (prob, a, plan, fill, b), E, inf in zip(items, Es, infos):
        for r in range(2):
            assert inf[r]["status"] == 0 and inf[r]["r_rel"] <= 1.05e-3, inf[r]
        solo = plan.solve(b, tol=1e-3, maxit=3000, method=psfd.PSFD_GMRES, restart=30)
        torch.cuda.synchronize()
        assert rel_l2(E.cpu(), solo["E"].cpu()) < 1e-6
    # one member against the FP64 oracle: its true residual is the solver's
    prob, a, plan, fill, b = items[1]
    g, fill_o = oracle_setup(prob, a)
    for r, pol in enumerate(prob.pols):
        bo = O.source_b(g, fill_o, pol)
        assert O.rel_residual(g, Es[1][r].cpu().to(torch.complex128), fill_o, bo) < 1.1e-3


@pytest.mark.parametrize("nz", [16, 32, 48, 64, 128])
def test_every_tuned_tile_gives_the_same_operator(nz):
    from paper_2607_25330_b300 import psfd
    prob = problem(32, 32, nz, theta=6.0, pols=[0])
    plan = psfd.Plan(prob)
    fill = plan.mask_fill(torch.from_numpy(I.mask_for(prob, 1)), prob.zprofile())
    plan.background(prob.stack(), fill, prob.pols)
    x = torch.from_numpy(I.random_field(plan.shape, 3)).to(torch.complex64).cuda()
    T = plan.autotune()
    assert T in (2, 4, 8)
    ref = plan.apply(x, flags=psfd.PSFD_PRECOND).cpu()
    g, fill_o = oracle_setup(prob, I.mask_for(prob, 1))
    assert rel_l2(ref[0], O.apply_A(g, O.apply_M(g, x[0].cpu().to(torch.complex128)), fill_o)) < 1e-4


def test_batched_layered_solves_reach_1e6():
    """Config-3 style batch (uneven lateral size and depth, 4/6/8 deg, TE + TM) with the layered
    preconditioner and FP64 refinement: every right-hand side reaches 1e-6 in its FP64 residual,
    with BiCGSTAB, and the batch equals the solo solves."""
    from paper_2607_25330_b300 import psfd
    specs = [(32, 32, 4.0, 1), (64, 48, 6.0, 2), (96, 32, 8.0, 3), (64, 64, 4.0, 4), (128, 64, 6.0, 6)]
    items = [make(*s) for s in specs]
    for it in items:
        with torch.cuda.stream(it[2].stream):
            it[2].layered_build()
    plans = [it[2] for it in items]
    bs = [it[4] for it in items]
    Es, infos = psfd.solve_batched(plans, bs, tol=1e-6, maxit=600, method=psfd.PSFD_BICGSTAB,
                                   precond=psfd.PC_LAYERED, refine=True)
    torch.cuda.synchronize()
    for (prob, a, plan, fill, b), E, inf in zip(items, Es, infos):
        for r in range(2):
            assert inf[r]["status"] == 0 and inf[r]["r_rel"] <= 1e-6 and inf[r]["iters"] <= 100, inf[r]
        solo = plan.solve_ex(b, tol=1e-6, maxit=600, method=psfd.PSFD_BICGSTAB, precond=psfd.PC_LAYERED)
        torch.cuda.synchronize()
        assert rel_l2(E.cpu(), solo["E"].cpu()) < 1e-6
    prob, a, plan, fill, b = items[4]
    g, fill_o = oracle_setup(prob, a)
    for r, pol in enumerate(prob.pols):
        bo = O.source_b(g, fill_o, pol)
        assert O.rel_residual(g, Es[4][r].cpu().to(torch.complex128), fill_o, bo) < 3e-6


_FIRST_USE = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2607_25330_b300 import inputs as I
from paper_2607_25330_b300 import psfd
from tests.helpers import problem
plans, bs = [], []
for k in range(8):
    prob = problem(64, 64, 32, theta=4.0 + k % 3, pols=[0, 1])
    pl = psfd.Plan(prob, stream=torch.cuda.Stream())
    pl.layered_storage(True)
    with torch.cuda.stream(pl.stream):
        fill = pl.mask_fill(torch.from_numpy(I.mask_for(prob, 50 + k)).cuda(), prob.zprofile())
        bs.append(pl.background(prob.stack(), fill, prob.pols))
    pl.layered_build()
    plans.append(pl)
torch.cuda.synchronize()
Es, infos = psfd.solve_batched(plans, bs, tol=1e-6, maxit=400, method=psfd.PSFD_BICGSTAB, precond=2,
                               refine=True, inner_tol=1e-3, nworkers=8)
assert all(i["status"] == 0 for inf in infos for i in inf), infos
print("ok")
"""


def test_first_use_from_several_host_threads():
    """A fresh process whose first applies of the layered P (the tensor-core pipeline, which needs a
    shared-memory attribute set once) come from eight host threads at once: the one-time set-up
    completes before any thread launches."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_USE, root], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]
