"""Pins of the oracle's factorised FNO (Sec. 2.1, Eqs. 1-5) and physics loss (Eq. loss)."""
import math

import numpy as np
import pytest
import torch

from oracle import fno as F
from oracle import krylov as K
from oracle import psfd as O
from paper_2607_25330_b300 import inputs as I

F64 = torch.float64


def test_gelu_is_the_erf_form():
    xs = [-4.0, -1.3, -0.2, 0.0, 0.7, 2.5]
    out = F.gelu(torch.tensor(xs, dtype=F64))
    for x, y in zip(xs, out.tolist()):
        assert abs(y - 0.5 * x * (1 + math.erf(x / math.sqrt(2)))) < 1e-15


def _dft_lowpass(n, m):
    """Explicit DFT-matrix projector onto the centred modes k = -m/2 .. m/2-1 (real part taken later)."""
    j = np.arange(n)
    ks = np.arange(-(m // 2), m - m // 2)
    Fm = np.exp(-2j * np.pi * np.outer(ks, j) / n)            # (m, n)
    return Fm.conj().T @ Fm / n                                # (n, n)


def test_identity_lateral_kernel_is_a_lowpass_projection():
    """Eq. 2 with K_oi(kx,ky) = delta_oi on the retained modes is Re(P_y v P_x^T), P the DFT low-pass."""
    B, dv, nz, ny, nx, m = 1, 3, 2, 12, 10, 6
    rng = np.random.default_rng(0)
    v = torch.from_numpy(rng.standard_normal((B, dv, nz, ny, nx)))
    Kxy = torch.zeros(m, m, dv, dv, dtype=torch.complex128)
    for i in range(dv):
        Kxy[:, :, i, i] = 1.0
    out = F.spectral_xy(v, Kxy, mix_bf16=False).numpy()
    Py, Px = _dft_lowpass(ny, m), _dft_lowpass(nx, m)
    ref = np.real(np.einsum("ab,...bc,dc->...ad", Py, v.numpy().astype(complex), Px))
    assert np.max(np.abs(out - ref)) < 1e-13


def test_identity_axial_kernel_is_a_lowpass_projection():
    B, dv, nz, ny, nx, m = 2, 2, 16, 3, 2, 6
    rng = np.random.default_rng(1)
    u = torch.from_numpy(rng.standard_normal((B, dv, nz, ny, nx)))
    Kz = torch.zeros(m, dv, dv, dtype=torch.complex128)
    for i in range(dv):
        Kz[:, i, i] = 1.0
    out = F.spectral_z(u, Kz, mix_bf16=False).numpy()
    Pz = _dft_lowpass(nz, m)
    ref = np.real(np.einsum("ab,...bcd->...acd", Pz, u.numpy().astype(complex)))
    assert np.max(np.abs(out - ref)) < 1e-13


def test_channel_mixing_is_per_mode_matrix_product():
    """A single retained mode with a random kernel: output = Re(F^-1 [K V]) evaluated by hand."""
    B, dv, nz, ny, nx = 1, 2, 1, 4, 4
    rng = np.random.default_rng(2)
    v = rng.standard_normal((B, dv, nz, ny, nx))
    m = 2
    Kxy = np.zeros((m, m, dv, dv), complex)
    Kxy[1, 1] = rng.standard_normal((dv, dv)) + 1j * rng.standard_normal((dv, dv))   # mode (0, 0)
    out = F.spectral_xy(torch.from_numpy(v), torch.from_numpy(Kxy), False).numpy()
    mean = v.mean(axis=(-2, -1))                                                        # DC / N
    ref = np.real(np.einsum("oi,biz->boz", Kxy[1, 1], mean))[..., None, None] * np.ones((ny, nx))
    assert np.max(np.abs(out - ref)) < 1e-14


def test_zero_operator_weights_reduce_to_lift_and_projection():
    S = I.FNOShape(dv=4, dh=6, layers=2, mx=4, my=4, mz=4, dq=5)
    w = I.fno_weights(S, 3)
    for k in ("kxy", "kz", "w2", "b2"):
        w[k] = np.zeros_like(w[k])
    a = torch.from_numpy(np.random.default_rng(4).random((1, 4, 6, 8)))
    E, hid = F.forward(w, a, return_hidden=True)
    for h in hid[1:]:
        assert torch.allclose(h, hid[0], rtol=0, atol=0)


def test_bf16_rounding_is_round_to_nearest_even():
    vals = torch.tensor([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -7 + 2 ** -8, -3.0 - 2 ** -7], dtype=F64)
    out = F._bf16(vals).tolist()
    assert out == [1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -3.0]


def test_spectral_upsampling_is_exact_for_band_limited_fields():
    nz0, ny0, nx0, nz, ny, nx = 4, 6, 8, 8, 12, 16
    def field(nz, ny, nx):
        z = np.arange(nz)[:, None, None] / nz
        y = np.arange(ny)[None, :, None] / ny
        x = np.arange(nx)[None, None, :] / nx
        return np.exp(2j * np.pi * (1 * x - 2 * y + 1 * z)) + 0.5 * np.exp(2j * np.pi * (-3 * x + 1 * z))
    out = F.spectral_upsample(torch.from_numpy(field(nz0, ny0, nx0)), nz, ny, nx).numpy()
    assert np.max(np.abs(out - field(nz, ny, nx))) < 1e-13


def test_loss_gradient_matches_central_differences():
    """dJ/dE from autograd against central finite differences of Eq. loss (tiny grid)."""
    p = I.Problem(nx=4, ny=4, nz=8, dx=2.0, dy=2.0, dz=2.0, theta_deg=6.0, pml_planes=2, z_ml=2,
                  abs_intervals=3.0, cap=True)
    g = O.Grid(p.to_dict(), I.multilayer_stack(True))
    a = I.manhattan_mask(4, 4, np.random.default_rng(3), nrect=(2, 3), edge=(1, 2))
    fill = O.fill_fraction(a, p.zprofile(), 1.0)
    b = O.source_b(g, fill, 0)
    A = lambda E: O.apply_A(g, E, fill)
    E = torch.from_numpy(I.random_field(g.shape, 5) * 0.3).requires_grad_(True)
    J = F.loss(A, E, b)
    J.backward()
    grad = E.grad.detach()
    rng = np.random.default_rng(6)
    for _ in range(3):
        d = torch.from_numpy(rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
        h = 1e-6
        with torch.no_grad():
            fd = (F.loss(A, E + h * d, b) - F.loss(A, E - h * d, b)) / (2 * h)
        # torch's complex gradient g satisfies dJ = Re <g, dE>
        lin = float(torch.vdot(grad.flatten(), d.flatten()).real)
        assert abs(float(fd) - lin) < 1e-6 * max(1.0, abs(lin))
    # and it equals the adjoint formula 2/N [A^H r + lam A^H F3^H (w^2 F3 r)]
    r = (A(E) - b).detach()
    N = g.N
    nu = torch.sqrt(torch.fft.fftfreq(g.nz, dtype=F64)[:, None, None] ** 2
                    + torch.fft.fftfreq(g.ny, dtype=F64)[None, :, None] ** 2
                    + torch.fft.fftfreq(g.nx, dtype=F64)[None, None, :] ** 2)
    w2 = (1.0 + nu) ** 2
    hf = torch.fft.ifftn(w2 * torch.fft.fftn(r, dim=(-3, -2, -1), norm="ortho"), dim=(-3, -2, -1), norm="ortho")
    adj = 2.0 / N * (O.apply_AH(g, r, fill) + 0.1 * O.apply_AH(g, hf, fill))
    assert float((adj - grad).abs().max()) < 1e-12 * float(grad.abs().max())


def _tiny_net(seed=31):
    S = I.FNOShape(dv=4, dh=6, layers=2, mx=4, my=4, mz=2, dq=5)
    w = I.fno_weights(S, seed, spectral_scale=8.0)
    return S, {k: torch.from_numpy(np.asarray(v)).to(torch.complex128 if np.iscomplexobj(v) else F64)
               for k, v in w.items()}


def test_network_parameter_gradients_match_central_differences():
    """Autograd through the float64 network (Eqs. 1-5) against central differences of J = Re<c, E>."""
    S, w = _tiny_net()
    a = torch.from_numpy(np.random.default_rng(8).random((1, 4, 8, 6)))
    c = torch.from_numpy(np.random.default_rng(9).standard_normal((1, 3, 4, 8, 6))
                         + 1j * np.random.default_rng(10).standard_normal((1, 3, 4, 8, 6)))
    J = lambda ww: float((c.conj() * F.forward(ww, a, mix_bf16=False)).real.sum())
    params = {k: v.clone().requires_grad_(True) for k, v in w.items()}
    (c.conj() * F.forward(params, a, mix_bf16=False)).real.sum().backward()
    rng = np.random.default_rng(11)
    h = 1e-6
    for name in ("lift_w", "lift_b", "kxy", "kz", "w1", "b2", "q1", "qb2"):
        g = params[name].grad
        for _ in range(2):
            idx = tuple(int(rng.integers(0, s)) for s in w[name].shape)
            for unit in ((1.0, 1j) if w[name].is_complex() else (1.0,)):
                wp = {k: v.clone() for k, v in w.items()}
                wm = {k: v.clone() for k, v in w.items()}
                wp[name][idx] += h * unit
                wm[name][idx] -= h * unit
                fd = (J(wp) - J(wm)) / (2 * h)
                # torch's gradient of a complex parameter is dJ/dRe + i dJ/dIm
                lin = float(g[idx].real) if unit == 1.0 else float(g[idx].imag)
                assert abs(fd - lin) < 1e-6 * max(1.0, abs(lin)), (name, idx, unit, fd, lin)


def test_bf16_mixing_gradient_is_straight_through():
    """With mix_bf16 the forward uses rounded operands; the gradient is the float64 chain rule
    evaluated at the rounded operands (dK = dU conj(bf16 V), dV = bf16(K)^H dU)."""
    rng = np.random.default_rng(12)
    K = torch.from_numpy(rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))).requires_grad_(True)
    V = torch.from_numpy(rng.standard_normal((3, 5)) + 1j * rng.standard_normal((3, 5))).requires_grad_(True)
    dU = torch.from_numpy(rng.standard_normal((3, 5)) + 1j * rng.standard_normal((3, 5)))
    U = F._bf16(K) @ F._bf16(V)
    # forward: exactly the product of the rounded operands
    Kr = torch.complex(K.real.detach().to(torch.bfloat16).to(F64), K.imag.detach().to(torch.bfloat16).to(F64))
    Vr = torch.complex(V.real.detach().to(torch.bfloat16).to(F64), V.imag.detach().to(torch.bfloat16).to(F64))
    assert torch.equal(U.detach(), Kr @ Vr)
    (dU.conj() * U).real.sum().backward()
    # the same products with the rounded values as plain float64 leaves
    Kl, Vl = Kr.clone().requires_grad_(True), Vr.clone().requires_grad_(True)
    (dU.conj() * (Kl @ Vl)).real.sum().backward()
    assert torch.allclose(K.grad, Kl.grad, rtol=0, atol=1e-14)
    assert torch.allclose(V.grad, Vl.grad, rtol=0, atol=1e-14)
