"""Oracle: factorised Fourier neural operator and physics-informed loss (float64 CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Forward pass, Sec. 2.1:
  v0 = lift([a, x, y, z])                                  (pointwise linear, 4 -> d_v)
  for each layer l:
    u_xy = Re F2^-1 [ sum_i K_xy[o,i](kx,ky) F2 v_i ]      (Eq. 2, per z-slice, retained
                                                            kx, ky in [-m/2, m/2-1])
    u_z  = Re F1^-1 [ sum_i K_z[o,i](kz) F1 u_xy,i ]        (Eq. 3, along z, kz in [-mz/2, mz/2-1])
    v   <- v + s_l( W2 gelu(W1 (u_xy + u_z) + b1) + b2 )    (Eq. 4; s_l = GELU except last layer)
  E = proj(v): d_v -> d_q -> 6 reals = (Re, Im) of (Ex, Ey, Ez), GELU between.
F2 / F1 are unnormalised forward DFTs and 1/N inverse DFTs; GELU is the exact
erf form.  The retained-mode tables hold k = -m/2 .. m/2-1 in that (centred) order.

``mix_bf16=True`` rounds both operands of the per-mode channel mixing to
bfloat16 (round to nearest even) before the float64 accumulation: the
arithmetic the workload prescribes for the mixing, done exactly.  Gradients
(torch autograd through this file) pass the rounding straight through.

Loss, Eq. loss:
  J = (1/N) sum_a ||r_a||^2 + (lambda_hf/N) sum_a || w(nu) F3[r_a] ||^2,
  r = A E - b, w = w0 + eta_hf |nu|, nu in cycles per sample, F3 unitary.
The paper does not give lambda_hf, w0, eta_hf or the normalisation of F3;
defaults are lambda_hf = 0.1, w0 = 1, eta_hf = 1 and the unitary DFT.

Parity pins (tests/test_oracle_fno.py): a layer whose kernels are the
identity on the retained modes equals an explicit low-pass projection written
with a DFT matrix; zero spectral and MLP weights leave the lifted field
unchanged; GELU against math.erf; loss gradients against central finite
differences; parameter gradients of the network (float64 mixing) against
central finite differences.
"""
from __future__ import annotations

import math
from typing import Dict

import torch

F64 = torch.float64
C128 = torch.complex128


def gelu(x: torch.Tensor) -> torch.Tensor:
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def kept_indices(n: int, m: int) -> torch.Tensor:
    """FFT-order indices of the centred modes k = -m/2 .. m/2-1 (all modes if m >= n)."""
    m = min(m, n)
    ks = torch.arange(-(m // 2), m - m // 2)
    return torch.remainder(ks, n)


def table_rows(n: int, m: int) -> torch.Tensor:
    """Rows of a centred mode table (k = -m/2 .. m/2-1) matching kept_indices(n, m)."""
    mm = min(m, n)
    return torch.arange(-(mm // 2), mm - mm // 2) + m // 2


def _round_bf16(x: torch.Tensor) -> torch.Tensor:
    return x.to(torch.bfloat16).to(F64)


def _bf16(x: torch.Tensor) -> torch.Tensor:
    """Round to bfloat16 (nearest even); under autograd the rounding is passed straight through.

    x + (round(x) - x) equals round(x) exactly in float64 (the difference is exact),
    and the detached difference makes the derivative the identity, so that
    gradients of the mixing are dK = dU conj(bf16(V)) and dV = bf16(K)^H dU.
    """
    if x.is_complex():
        re, im = x.real, x.imag
        return torch.complex(re + (_round_bf16(re) - re).detach(), im + (_round_bf16(im) - im).detach())
    return x + (_round_bf16(x) - x).detach()


def _t(w, dtype=F64):
    return torch.as_tensor(w).to(dtype)


def coords(nz: int, ny: int, nx: int):
    z = torch.arange(nz, dtype=F64) / nz
    y = torch.arange(ny, dtype=F64) / ny
    x = torch.arange(nx, dtype=F64) / nx
    Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def spectral_xy(v: torch.Tensor, K: torch.Tensor, mix_bf16: bool) -> torch.Tensor:
    """Eq. 2: v (B, dv, nz, ny, nx) real, K (my, mx, out, in) complex -> (B, dv, nz, ny, nx) real."""
    B, dv, nz, ny, nx = v.shape
    my, mx = K.shape[0], K.shape[1]
    iy = kept_indices(ny, my)
    ix = kept_indices(nx, mx)
    sel_y = table_rows(ny, my)
    sel_x = table_rows(nx, mx)
    V = torch.fft.fft2(v.to(C128), dim=(-2, -1))[..., iy[:, None], ix[None, :]]   # (B, dv, nz, my', mx')
    Ks = K.to(C128)[sel_y][:, sel_x]                                              # (my', mx', out, in)
    if mix_bf16:
        V = _bf16(V)
        Ks = _bf16(Ks)
    U = torch.einsum("yxoi,bizyx->bozyx", Ks, V)
    full = torch.zeros(B, dv, nz, ny, nx, dtype=C128)
    full[..., iy[:, None], ix[None, :]] = U
    return torch.fft.ifft2(full, dim=(-2, -1)).real


def spectral_z(u: torch.Tensor, K: torch.Tensor, mix_bf16: bool) -> torch.Tensor:
    """Eq. 3: u (B, dv, nz, ny, nx) real, K (mz, out, in) complex."""
    B, dv, nz, ny, nx = u.shape
    mz = K.shape[0]
    iz = kept_indices(nz, mz)
    sel = table_rows(nz, mz)
    W = torch.fft.fft(u.to(C128), dim=2)[:, :, iz]                                # (B, dv, mz', ny, nx)
    Ks = K.to(C128)[sel]
    if mix_bf16:
        W = _bf16(W)
        Ks = _bf16(Ks)
    U = torch.einsum("zoi,bizyx->bozyx", Ks, W)
    full = torch.zeros(B, dv, nz, ny, nx, dtype=C128)
    full[:, :, iz] = U
    return torch.fft.ifft(full, dim=2).real


def pointwise(W: torch.Tensor, b: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Channel-mixing linear map on (B, C, ...) fields."""
    return torch.einsum("oi,bi...->bo...", W, x) + b.reshape((1, -1) + (1,) * (x.dim() - 2))


def forward(w: Dict, a: torch.Tensor, mix_bf16: bool = False, return_hidden: bool = False):
    """G_theta: a (B, nz, ny, nx) in [0,1] -> E (B, 3, nz, ny, nx) complex (Eq. 5)."""
    a = _t(a)
    B, nz, ny, nx = a.shape
    X, Y, Z = coords(nz, ny, nx)
    inp = torch.stack([a, X.expand(B, -1, -1, -1), Y.expand(B, -1, -1, -1), Z.expand(B, -1, -1, -1)], dim=1)
    v = pointwise(_t(w["lift_w"]), _t(w["lift_b"]), inp)
    L = _t(w["w1"]).shape[0]
    hidden = [v]
    for l in range(L):
        uxy = spectral_xy(v, _t(w["kxy"][l], C128), mix_bf16)
        uz = spectral_z(uxy, _t(w["kz"][l], C128), mix_bf16)
        h = gelu(pointwise(_t(w["w1"][l]), _t(w["b1"][l]), uxy + uz))
        o = pointwise(_t(w["w2"][l]), _t(w["b2"][l]), h)
        v = v + (gelu(o) if l < L - 1 else o)
        hidden.append(v)
    q = gelu(pointwise(_t(w["q1"]), _t(w["qb1"]), v))
    o6 = pointwise(_t(w["q2"]), _t(w["qb2"]), q)                 # (B, 6, ...)
    E = torch.complex(o6[:, 0::2], o6[:, 1::2])                  # (B, 3, nz, ny, nx)
    if return_hidden:
        return E, hidden
    return E


def spectral_upsample(E: torch.Tensor, nz: int, ny: int, nx: int) -> torch.Tensor:
    """Zero-pad the 3-D spectrum of E (..., nz0, ny0, nx0) to (nz, ny, nx), amplitude preserving."""
    nz0, ny0, nx0 = E.shape[-3:]
    F = torch.fft.fftn(E.to(C128), dim=(-3, -2, -1))
    out = torch.zeros(E.shape[:-3] + (nz, ny, nx), dtype=C128)
    iz0, iy0, ix0 = kept_indices(nz0, nz0), kept_indices(ny0, ny0), kept_indices(nx0, nx0)
    iz1 = torch.remainder(torch.arange(-(nz0 // 2), nz0 - nz0 // 2), nz)
    iy1 = torch.remainder(torch.arange(-(ny0 // 2), ny0 - ny0 // 2), ny)
    ix1 = torch.remainder(torch.arange(-(nx0 // 2), nx0 - nx0 // 2), nx)
    out[..., iz1[:, None, None], iy1[None, :, None], ix1[None, None, :]] = \
        F[..., iz0[:, None, None], iy0[None, :, None], ix0[None, None, :]]
    scale = (nz * ny * nx) / (nz0 * ny0 * nx0)
    return torch.fft.ifftn(out, dim=(-3, -2, -1)) * scale


def loss(A, E: torch.Tensor, b: torch.Tensor, lam_hf: float = 0.1, w0: float = 1.0, eta_hf: float = 1.0):
    """Eq. loss for one sample: E, b (3, nz, ny, nx); A maps a field to A field."""
    r = A(E) - b
    nz, ny, nx = r.shape[-3:]
    N = nz * ny * nx
    nu = torch.sqrt(torch.fft.fftfreq(nz, dtype=F64)[:, None, None] ** 2
                    + torch.fft.fftfreq(ny, dtype=F64)[None, :, None] ** 2
                    + torch.fft.fftfreq(nx, dtype=F64)[None, None, :] ** 2)
    wgt = w0 + eta_hf * nu
    R3 = torch.fft.fftn(r, dim=(-3, -2, -1), norm="ortho")
    return (r.abs() ** 2).sum() / N + lam_hf * ((wgt * R3.abs()) ** 2).sum() / N
