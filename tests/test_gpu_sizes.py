"""GPU parity at the lateral sizes the large workloads run (256^2, 512^2), of the FP64
operator apply, and of the FNO forward with and without the bfloat16 mixing.

Every comparison goes through the C ABI against the FP64 oracle on the same seeded inputs.
Tolerances: complex64 operator outputs relative L2 1e-4; the FP64 apply (the operator of
the refinement residual, Sec. 2.2 with Eq. relative_residual) 1e-10; the FNO forward with
float32 mixing operands 1e-4 against the float64 network (Sec. 2.1, Eqs. 2-5).  The
measured errors are printed (pytest -s shows them).
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import fno as F
from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I
from tests.helpers import oracle_setup, problem, rel_l2

pytestmark = pytest.mark.gpu
TOL_C64 = 1e-4
TOL_FP64 = 1e-10


def setup(nx, ny, nz, theta, nrhs, seed=2, kind=None):
    from paper_2607_25330_b300 import psfd
    prob = problem(nx, ny, nz, theta=theta, pols=[i % 2 for i in range(nrhs)])
    a = I.mask_for(prob, seed, kind)
    g, fill_o = oracle_setup(prob, a)
    plan = psfd.Plan(prob, nrhs=nrhs)
    fill = plan.mask_fill(torch.from_numpy(a), prob.zprofile())
    plan.background(prob.stack(), fill, prob.pols)
    return prob, g, fill_o, plan, fill


@pytest.mark.parametrize("flags", [0, 1, 4])
def test_apply_256x256_matches_oracle(flags):
    """A, A M and A^H on a 256^2 lateral grid (the largest lateral size of the batched workload)."""
    prob, g, fill_o, plan, fill = setup(256, 256, 16, 6.0, 2)
    assert prob.zprofile().sum() > 0 and float(fill_o.abs().max()) > 0.5
    x = torch.from_numpy(I.random_field(plan.shape, 17)).to(torch.complex64)
    y = plan.apply(x.cuda(), flags=flags).cpu()
    for r in range(plan.nrhs):
        xr = x[r].to(torch.complex128)
        if flags == 4:
            ref = O.apply_AH(g, xr, fill_o)
        else:
            ref = O.apply_A(g, O.apply_M(g, xr) if flags else xr, fill_o)
        e = rel_l2(y[r], ref)
        print(f"256x256x16 flags {flags} rhs {r}: rel L2 {e:.2e}")
        assert e < TOL_C64


@pytest.mark.parametrize("flags", [0, 4])
def test_apply_512x512_with_contrast_matches_oracle(flags):
    """A and A^H on a 512^2 lateral grid with a dense Manhattan absorber (the fine-grid size)."""
    prob, g, fill_o, plan, fill = setup(512, 512, 16, 6.0, 1, kind="manhattan_dense")
    x = torch.from_numpy(I.random_field(plan.shape, 18)).to(torch.complex64)
    y = plan.apply(x.cuda(), flags=flags).cpu()
    xr = x[0].to(torch.complex128)
    ref = O.apply_AH(g, xr, fill_o) if flags == 4 else O.apply_A(g, xr, fill_o)
    # the contrast term alone must be resolved too, not only the dominant curl-curl part
    contrast = ref - (O.curlcurl(g, xr, adjoint_form=(flags == 4)) - g.k0 ** 2 * xr)
    assert float(torch.linalg.vector_norm(contrast) / torch.linalg.vector_norm(ref)) > 1e-3
    e = rel_l2(y[0], ref)
    ec = float(torch.linalg.vector_norm(y[0].to(torch.complex128) - ref) / torch.linalg.vector_norm(contrast))
    print(f"512x512x16 flags {flags}: rel L2 {e:.2e}, error / contrast term {ec:.2e}")
    assert e < TOL_C64
    assert ec < 1e-2


FP64_GRIDS = [  # (nx, ny, nz, theta, nrhs): every axial length, lateral 16 ... 512
    (32, 32, 16, 6.0, 1),
    (16, 32, 32, 8.0, 2),
    (64, 16, 48, 4.0, 1),
    (96, 96, 64, 6.0, 1),
    (128, 64, 96, 6.0, 1),
    (16, 16, 128, 5.0, 2),
    (256, 256, 16, 6.0, 1),
    (512, 512, 16, 6.0, 1),
]


@pytest.mark.parametrize("grid", FP64_GRIDS)
def test_apply64_matches_oracle(grid):
    """The FP64 operator apply of the refinement residual, element by element, real space and HYBRID.

    The fill is given to both sides directly (psfd_background takes any fill): the binary layout
    extruded with the absorber's z profile, exact in float32, so that the float32 storage of a
    smoothed fill does not enter an FP64 comparison."""
    from paper_2607_25330_b300 import psfd
    nx, ny, nz, theta, nrhs = grid
    prob = problem(nx, ny, nz, theta=theta, pols=[i % 2 for i in range(nrhs)])
    a = I.mask_for(prob, 2)
    fill_np = prob.zprofile()[:, None, None] * a[None].astype(np.float64)
    assert np.array_equal(fill_np.astype(np.float32).astype(np.float64), fill_np)
    fill_o = torch.from_numpy(fill_np)
    g = O.Grid(prob.to_dict(), prob.stack())
    plan = psfd.Plan(prob, nrhs=nrhs)
    fill = torch.from_numpy(fill_np.astype(np.float32)).cuda()
    plan.background(prob.stack(), fill, prob.pols)
    x = torch.from_numpy(I.random_field(plan.shape, 19))                     # complex128
    y = plan.apply64(x.cuda()).cpu()
    xh = torch.fft.fft2(x, norm="ortho").contiguous()
    yh = plan.apply64(xh.cuda(), flags=psfd.PSFD_HYBRID).cpu()
    for r in range(plan.nrhs):
        ref = O.apply_A(g, x[r], fill_o)
        e = rel_l2(y[r], ref)
        eh = rel_l2(yh[r], torch.fft.fft2(ref, norm="ortho"))
        emax = float((y[r] - ref).abs().max() / ref.abs().max())
        print(f"FP64 apply {grid} rhs {r}: rel L2 {e:.2e} (HYBRID {eh:.2e}), max-entry {emax:.2e}")
        assert e < TOL_FP64 and eh < TOL_FP64
        assert emax < 10 * TOL_FP64


def _device_weights(w):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda().contiguous() for k, v in w.items()}


def _flip_sensitivity(w, a, rel=2.0 ** -22, seed=3):
    """How far the bf16-mixing network moves when its mixing operands carry float32-level noise
    before the rounding (oracle only): the size of a deviation that flipped rounding decisions cause."""
    gen = torch.Generator().manual_seed(seed)
    orig = F._round_bf16

    def noisy(x):
        n = (torch.rand(x.shape, generator=gen, dtype=torch.float64) * 2 - 1) * rel
        return orig(x * (1 + n))
    try:
        F._round_bf16 = noisy
        E1 = F.forward(w, a, mix_bf16=True)
    finally:
        F._round_bf16 = orig
    return rel_l2(E1, F.forward(w, a, mix_bf16=True))


@pytest.mark.parametrize("dims", [(2, 32, 32, 16), (1, 64, 32, 32)])
def test_fno_forward_float32_mixing_matches_float64_network(dims):
    """Without the bf16 rounding (PSFD_MIX_FP32=1) the GPU forward equals the float64 network to 1e-4:
    every other step (FFTs, mode truncation, lift, MLP, GELU, projection) is exact to float32 level.
    With the rounding, the GPU's deviation from the oracle's bf16 network is of the size that float32
    noise before the rounding produces in the oracle itself (flipped rounding decisions)."""
    from paper_2607_25330_b300 import psfd
    B, nx, ny, nz = dims
    S = I.FNOShape()
    w = I.fno_weights(S, 21, spectral_scale=4.0)
    a = np.random.default_rng(5).random((B, nz, ny, nx)).astype(np.float32)
    ws = psfd.fno_struct(_device_weights(w), S)
    at = torch.from_numpy(a).cuda()
    old = os.environ.get("PSFD_MIX_FP32")
    os.environ["PSFD_MIX_FP32"] = "1"
    try:
        E32 = psfd.fno_forward(ws, at).cpu()
    finally:
        if old is None:
            del os.environ["PSFD_MIX_FP32"]
        else:
            os.environ["PSFD_MIX_FP32"] = old
    Ebf = psfd.fno_forward(ws, at).cpu()
    ad = torch.from_numpy(a).double()
    ref64 = F.forward(w, ad, mix_bf16=False)
    refbf = F.forward(w, ad, mix_bf16=True)
    e32 = rel_l2(E32, ref64)
    ebf = rel_l2(Ebf, refbf)
    flip = _flip_sensitivity(w, ad)
    print(f"FNO {dims}: float32 mixing vs float64 network {e32:.2e}; bf16 mixing vs bf16 oracle {ebf:.2e}; "
          f"oracle moved by float32-level noise before rounding {flip:.2e}")
    assert e32 < 1e-4
    assert ebf < max(4.0 * flip, 1e-4)
