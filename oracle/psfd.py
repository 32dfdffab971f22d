"""Oracle: background-decomposed PSFD operator in complex128 on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (the paper defers the discretisation details to its companion
PSFD paper; these are the readings used throughout):

* time dependence exp(-i w t); plane waves exp(+i k.r); z points up; the
  illumination comes from +z and travels towards -z onto the multilayer, whose
  top face is the plane z_ml (Sec. 2.2).
* lateral directions are periodic with a Bloch shift: fields are envelopes,
  physical field = envelope * exp(i (kx_inc x + ky_inc y)); so d/dx ->
  i (k_xm + kx_inc) with k_xm = 2 pi m / (Nx dx) (Sec. 3, representable
  wavenumbers), m in FFT order, the Nyquist index -N/2 kept.
* the axial direction is a periodic FFT box that contains a PML at both ends:
  d/dz -> D_z = s(z)^-1 F_z^-1 (i k_z) F_z with s = 1 + i alpha (d/d_pml)^3
  and alpha = 4 ln(1/R0) / (2 k0 d_pml) (stretched-coordinate PML, Sec. 2.2).
  The two PMLs meet across the periodic wrap.  A z-stretch cannot attenuate a
  field that is constant in z (D_z annihilates it for any s), so a lateral
  Bloch mode near grazing, |k_par| ~ k0, would keep an undamped standing mode
  with the real eigenvalue |k_par|^2 - k0^2 ~ 0.  The PML is therefore backed
  by an absorbing layer, as a PML is backed by a terminating wall: on the
  outermost nb = max(1, npml / 4) planes at each end, eps_bg = 1 + i sigma with
  sigma = sigma_b ((nb - j) / nb)^2 on the j-th plane from the end (sigma_b =
  pml_backing), which the scattered field reaches only after the PML has
  attenuated every wave that is not near grazing.
* unknown: the scattered field E_s in the mask-only domain.  The multilayer
  enters through the reflection operator R (Sec. 2.2: up/down split, TE/TM
  split, transfer-matrix reflection, phase-matched propagation), applied to the
  tangential field at z_ml and linear in its argument, so
      A E = curl_s curl_s E - k0^2 E - k0^2 deps (E + R E)
      b   = k0^2 deps (E_inc + R E_inc)                 (Eq. bg_source)
  which is  L E - b  with L = curl curl - k0^2 eps (Eq.
  vector_helmholtz_operator) and eps = 1 + deps.
* R per lateral mode k_par: a_s = s_hat . E_par(z_ml), a_t = t_hat . E_par(z_ml),
  s_hat = (-ky, kx)/|k_par|, t_hat = k_par/|k_par| (s_hat = y, t_hat = x at
  k_par = 0); reflected tangential field r_s a_s s_hat + r_p a_t t_hat,
  E_z = -(k_par . E_par_refl)/k_z (upgoing, divergence free), profile
  exp(i k_z (z - z_ml)) for z >= z_ml and 0 below; k_z = sqrt(k0^2 - k_par^2)
  with Im k_z >= 0.  r_s, r_p are the ratios of reflected to incident
  tangential E of the stack (r_p therefore equals r_s at normal incidence).

Parity pins (tests/test_oracle_*.py): FFT-free plane-wave symbol of the
curl-curl operator, divergence and gradient identities, PML off -> periodic
operator, Fresnel / quarter-wave / lossless-stack closed forms for the
reflection coefficients, an independent transfer-matrix product, the blank-mask
invariant, the homogeneous absorber slab against the Airy formula and against
the reflection of [slab | multilayer], the adjoint identity and the dense
conjugate transpose, and the periodised Gaussian for the smoothing.  The
layered-background preconditioner (an addition to the paper's method): with a
laterally uniform fill it is the exact inverse of A; in the (s, t, z) basis of
every lateral mode its blocks do not couple E_s with (E_t, E_z).
"""
from __future__ import annotations

import cmath
import math
from typing import Dict, Optional, Sequence

import torch

C128 = torch.complex128
F64 = torch.float64


def sqrt_up(z: torch.Tensor) -> torch.Tensor:
    """Square root on the branch Im >= 0 (decaying / outgoing waves)."""
    r = torch.sqrt(z.to(C128))
    return torch.where(r.imag < 0, -r, r)


def fftfreq_k(n: int, d: float) -> torch.Tensor:
    """Angular wavenumbers 2 pi m / (n d) in FFT order (Nyquist at index n/2 as -n/2)."""
    return 2.0 * math.pi * torch.fft.fftfreq(n, d=d, dtype=F64)


class Grid:
    """Grid, illumination, PML and multilayer tables of one problem.

    ``p`` is a plain dict with the keys of ``paper_2607_25330_b300.inputs.Problem``;
    ``stack`` is {"n": [...], "d": [...], "n_sub": complex}, listed top to bottom.
    """

    def __init__(self, p: Dict, stack: Dict):
        self.nx, self.ny, self.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])
        self.dx, self.dy, self.dz = float(p["dx"]), float(p["dy"]), float(p["dz"])
        self.lam = float(p["lam"])
        self.k0 = 2.0 * math.pi / self.lam
        th = math.radians(float(p["theta_deg"]))
        ph = math.radians(float(p["phi_deg"]))
        self.theta, self.phi = th, ph
        self.kx_inc = self.k0 * math.sin(th) * math.cos(ph)
        self.ky_inc = self.k0 * math.sin(th) * math.sin(ph)
        self.kz_inc = self.k0 * math.cos(th)
        self.kx = fftfreq_k(self.nx, self.dx) + self.kx_inc
        self.ky = fftfreq_k(self.ny, self.dy) + self.ky_inc
        self.kz = fftfreq_k(self.nz, self.dz)
        self.KY, self.KX = torch.meshgrid(self.ky, self.kx, indexing="ij")   # (ny, nx)
        self.z_ml = int(p["z_ml"])
        self.eps_abs = complex(p["n_abs"]) ** 2
        self.deps_abs = self.eps_abs - 1.0
        # per-plane material contrast c[z] (deps = fill * c[z]); None: c[z] = eps_abs - 1
        self.plane_contrast = None
        # PML (stretched coordinate, cubic grading, both ends of the z box)
        npml = int(p["pml_planes"])
        self.sigma = torch.zeros(self.nz, dtype=F64)
        if npml > 0:
            dpml = npml * self.dz
            alpha = 4.0 * math.log(1.0 / float(p["pml_R0"])) / (2.0 * self.k0 * dpml)
            for k in range(self.nz):
                if k < npml:
                    d = (npml - k) * self.dz
                elif k >= self.nz - npml:
                    d = (k - (self.nz - npml - 1)) * self.dz
                else:
                    continue
                self.sigma[k] = alpha * (d / dpml) ** 3
        self.s = (1.0 + 1j * self.sigma).to(C128)
        self.s_inv = 1.0 / self.s
        # absorbing backing of the PML: eps_bg = 1 + i sigma(z) on the outermost nb = max(1, npml / 4)
        # planes at each end of the box (where the two PMLs meet across the periodic wrap), with
        # sigma = sigma_b ((nb - j) / nb)^2 on the j-th plane from the end (j = 0 outermost)
        self.backing = torch.zeros(self.nz, dtype=F64)
        sb = float(p.get("pml_backing", 0.0))
        if npml > 0 and sb > 0:
            nb = max(1, npml // 4)
            for j in range(nb):
                self.backing[j] = self.backing[self.nz - 1 - j] = sb * ((nb - j) / nb) ** 2
        self.eps_bg = (1.0 + 1j * self.backing).to(C128)
        # spectral damping (Eq. spectral_damping_mask)
        self.m_min = float(p["m_min"])
        self.k_ref = float(p["k_ref"]) if float(p["k_ref"]) > 0 else self.k0
        self.gamma = float(p["gamma"])
        self.damp_eps = float(p["damp_eps_rel"]) * self.k0 ** 2
        self.sigma_px = float(p["sigma_px"])
        # multilayer reflection per lateral mode
        kpar2 = self.KX ** 2 + self.KY ** 2
        self.kpar = torch.sqrt(kpar2)
        kz0 = sqrt_up(self.k0 ** 2 - kpar2 + 0j)
        if bool((kz0.abs() < 1e-9 * self.k0).any()):
            raise ValueError("a lateral mode sits exactly on the light cone (k_z = 0)")
        self.kz0 = kz0
        self.stack = stack
        self.rs = reflection_coefficient(kpar2, stack, self.k0, pol="s")
        self.rp = reflection_coefficient(kpar2, stack, self.k0, pol="p")
        small = self.kpar < 1e-12 * self.k0
        safe = torch.where(small, torch.ones_like(self.kpar), self.kpar)
        self.sx = torch.where(small, torch.zeros_like(self.kpar), -self.KY / safe).to(C128)
        self.sy = torch.where(small, torch.ones_like(self.kpar), self.KX / safe).to(C128)
        self.tx = torch.where(small, torch.ones_like(self.kpar), self.KX / safe).to(C128)
        self.ty = torch.where(small, torch.zeros_like(self.kpar), self.KY / safe).to(C128)
        zrel = (torch.arange(self.nz, dtype=F64) - self.z_ml) * self.dz
        prof = torch.exp(1j * kz0[None, :, :] * zrel[:, None, None].to(C128))
        self.prof = torch.where(zrel[:, None, None] >= 0, prof, torch.zeros_like(prof))  # (nz, ny, nx)

    @property
    def shape(self):
        return (3, self.nz, self.ny, self.nx)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz


# --------------------------------------------------------------------------- geometry

def gaussian_smooth(a_bin: torch.Tensor, sigma_px: float) -> torch.Tensor:
    """Periodic Gaussian smoothing of a 2-D binary indicator (Sec. 2.1 / Sec. 3).

    Spectral multiply by exp(-sigma^2 |kappa|^2 / 2), kappa in radians per pixel.
    """
    ny, nx = a_bin.shape
    kx = 2.0 * math.pi * torch.fft.fftfreq(nx, dtype=F64)
    ky = 2.0 * math.pi * torch.fft.fftfreq(ny, dtype=F64)
    g = torch.exp(-0.5 * sigma_px ** 2 * (ky[:, None] ** 2 + kx[None, :] ** 2))
    return torch.fft.ifft2(g * torch.fft.fft2(a_bin.to(F64))).real


def fill_fraction(a_bin, zprof, sigma_px: float) -> torch.Tensor:
    """Smoothed indicator extruded through the absorber: f[z, y, x] = zprof[z] * a(x, y)."""
    a = gaussian_smooth(torch.as_tensor(a_bin), sigma_px)
    return torch.as_tensor(zprof, dtype=F64)[:, None, None] * a[None, :, :]


# --------------------------------------------------------------------------- multilayer

def reflection_coefficient(kpar2: torch.Tensor, stack: Dict, k0: float, pol: str) -> torch.Tensor:
    """Reflection of the stack below z_ml seen from vacuum (Sec. 2.2, TMM response).

    Layers are combined from the substrate upwards with the Airy recursion
        G_{j-1} = (r_{j-1,j} + G_j e^{2 i kz_j d_j}) / (1 + r_{j-1,j} G_j e^{2 i kz_j d_j}),
    which is the transfer-matrix result written in a form that stays finite for
    evanescent modes.  Interface coefficients are ratios of tangential E:
        s: (kz_a - kz_b) / (kz_a + kz_b)
        p: (eps_a kz_b - eps_b kz_a) / (eps_b kz_a + eps_a kz_b).
    """
    eps = [complex(n) ** 2 for n in stack["n"]]
    d = [float(t) for t in stack["d"]]
    media = [1.0 + 0j] + eps + [complex(stack["n_sub"]) ** 2]
    kz = [sqrt_up(k0 ** 2 * e - kpar2 + 0j) for e in media]

    def r_iface(a: int, b: int) -> torch.Tensor:
        if pol == "s":
            return (kz[a] - kz[b]) / (kz[a] + kz[b])
        ea, eb = media[a], media[b]
        return (ea * kz[b] - eb * kz[a]) / (eb * kz[a] + ea * kz[b])

    nl = len(eps)
    G = r_iface(nl, nl + 1)                      # top of the substrate, seen from the last layer
    for j in range(nl, 0, -1):                   # layer j occupies media index j
        ph = torch.exp(2j * kz[j] * d[j - 1])
        r = r_iface(j - 1, j)
        G = (r + G * ph) / (1.0 + r * G * ph)
    return G


# --------------------------------------------------------------------------- operator

def _fft2(u):
    return torch.fft.fft2(u, dim=(-2, -1))


def _ifft2(u):
    return torch.fft.ifft2(u, dim=(-2, -1))


def _dz(g: Grid, u: torch.Tensor, adjoint_form: bool = False) -> torch.Tensor:
    """Stretched axial derivative along dim 0 of u (nz, ny, nx).

    D_z u = s^-1 F^-1 (i k_z F u); the adjoint form D~_z u = F^-1 (i k_z F (conj(s^-1) u))
    satisfies D_z^H = -D~_z.
    """
    ikz = (1j * g.kz).to(C128)[:, None, None]
    if adjoint_form:
        return torch.fft.ifft(ikz * torch.fft.fft(g.s_inv.conj()[:, None, None] * u, dim=0), dim=0)
    return g.s_inv[:, None, None] * torch.fft.ifft(ikz * torch.fft.fft(u, dim=0), dim=0)


def _curl_h(g: Grid, Eh: torch.Tensor, adjoint_form: bool = False) -> torch.Tensor:
    """Curl of a field given in the lateral-spectral domain (kx, ky, z)."""
    ikx = (1j * g.KX).to(C128)[None]
    iky = (1j * g.KY).to(C128)[None]
    ex, ey, ez = Eh[0], Eh[1], Eh[2]
    cx = iky[0] * ez - _dz(g, ey, adjoint_form)
    cy = _dz(g, ex, adjoint_form) - ikx[0] * ez
    cz = ikx[0] * ey - iky[0] * ex
    return torch.stack([cx, cy, cz])


def curlcurl(g: Grid, E: torch.Tensor, adjoint_form: bool = False) -> torch.Tensor:
    """curl_s curl_s E in real space (the derivative part of Eq. vector_helmholtz_operator)."""
    Eh = _fft2(E.to(C128))
    return _ifft2(_curl_h(g, _curl_h(g, Eh, adjoint_form), adjoint_form))


def _refl_matrix(g: Grid) -> torch.Tensor:
    """Per-mode 3x2 map from (E_x, E_y) at z_ml to the reflected vector at z_ml."""
    T = torch.zeros(g.ny, g.nx, 3, 2, dtype=C128)
    sx, sy, tx, ty = g.sx, g.sy, g.tx, g.ty
    T[..., 0, 0] = g.rs * sx * sx + g.rp * tx * tx
    T[..., 0, 1] = g.rs * sx * sy + g.rp * tx * ty
    T[..., 1, 0] = g.rs * sy * sx + g.rp * ty * tx
    T[..., 1, 1] = g.rs * sy * sy + g.rp * ty * ty
    KX, KY = g.KX.to(C128), g.KY.to(C128)
    T[..., 2, 0] = -(KX * T[..., 0, 0] + KY * T[..., 1, 0]) / g.kz0
    T[..., 2, 1] = -(KX * T[..., 0, 1] + KY * T[..., 1, 1]) / g.kz0
    return T


def reflect(g: Grid, E: torch.Tensor) -> torch.Tensor:
    """Multilayer-reflected field R E (Sec. 2.2, operator R_ml, linear part).

    Steps per lateral mode: tangential field at z_ml -> TE/TM split -> r_s, r_p
    -> divergence-free upgoing vector -> exp(i k_z (z - z_ml)) above z_ml.
    """
    e0 = _fft2(E[:2, g.z_ml].to(C128))                   # (2, ny, nx)
    ex, ey = e0[0], e0[1]
    a_s = g.sx * ex + g.sy * ey
    a_t = g.tx * ex + g.ty * ey
    rx = g.rs * a_s * g.sx + g.rp * a_t * g.tx
    ry = g.rs * a_s * g.sy + g.rp * a_t * g.ty
    rz = -(g.KX * rx + g.KY * ry) / g.kz0
    vec = torch.stack([rx, ry, rz])                      # (3, ny, nx)
    return _ifft2(vec[:, None, :, :] * g.prof[None])


def reflect_adjoint(g: Grid, U: torch.Tensor) -> torch.Tensor:
    """R^H: projection on the upgoing profile, conjugate-transposed 3x2 map, placed at z_ml."""
    Uh = _fft2(U.to(C128))                               # (3, nz, ny, nx)
    v = (g.prof.conj()[None] * Uh).sum(dim=1)            # (3, ny, nx)
    T = _refl_matrix(g)
    e = torch.einsum("yxab,ayx->byx", T.conj(), v)       # (2, ny, nx)
    out = torch.zeros(g.shape, dtype=C128)
    out[:2, g.z_ml] = _ifft2(e)
    return out


def deps_field(g: Grid, fill: torch.Tensor) -> torch.Tensor:
    """Permittivity contrast deps = eps - eps_bg = f * (eps_abs - 1) (Sec. 2.2), or f * c[z] with a
    per-plane material table (a layered structure meshed in the domain)."""
    if g.plane_contrast is None:
        return fill.to(C128) * g.deps_abs
    c = torch.as_tensor(g.plane_contrast, dtype=C128)
    return fill.to(C128) * c[:, None, None]


def apply_A(g: Grid, E: torch.Tensor, fill: torch.Tensor) -> torch.Tensor:
    """A E = curl_s curl_s E - k0^2 eps_bg E - k0^2 deps (E + R E)  (Eqs. bg_source,
    vector_helmholtz_operator); eps_bg = 1 except on the PML's absorbing backing."""
    E = E.to(C128)
    de = deps_field(g, fill)[None]
    ebg = g.eps_bg[None, :, None, None]
    return curlcurl(g, E) - g.k0 ** 2 * ebg * E - g.k0 ** 2 * de * (E + reflect(g, E))


def apply_AH(g: Grid, Y: torch.Tensor, fill: torch.Tensor) -> torch.Tensor:
    """Adjoint A^H Y = (curl~ curl~) Y - k0^2 conj(eps_bg) Y - k0^2 (I + R)^H (conj(deps) Y)."""
    Y = Y.to(C128)
    w = deps_field(g, fill).conj()[None] * Y
    ebg = g.eps_bg.conj()[None, :, None, None]
    return curlcurl(g, Y, adjoint_form=True) - g.k0 ** 2 * ebg * Y - g.k0 ** 2 * (w + reflect_adjoint(g, w))


def damping_multiplier(g: Grid) -> torch.Tensor:
    """m(k) of Eq. spectral_damping_mask on the 3-D grid (nz, ny, nx).

    |k|^2 = kx^2 + ky^2 + kz^2 with Bloch-shifted lateral and unstretched axial wavenumbers.
    """
    k2 = g.kz[:, None, None] ** 2 + g.KY[None] ** 2 + g.KX[None] ** 2
    damp = torch.where(k2.sqrt() <= g.k_ref, torch.ones_like(k2),
                       (g.k_ref ** 2 / (k2 + g.damp_eps)) ** g.gamma)
    return g.m_min + (1.0 - g.m_min) * damp


def apply_M(g: Grid, X: torch.Tensor) -> torch.Tensor:
    """Spectral damping M x, componentwise 3-D Fourier multiplier (Eq. spectral_damping_action)."""
    m = damping_multiplier(g).to(C128)
    return torch.fft.ifftn(m[None] * torch.fft.fftn(X.to(C128), dim=(1, 2, 3)), dim=(1, 2, 3))


def incident_field(g: Grid, pol: int) -> torch.Tensor:
    """Envelope of the incident plane wave, unit amplitude, phase reference at z_ml.

    TE (pol 0): E along s = (-sin phi, cos phi, 0); TM (pol 1): (cos th cos phi,
    cos th sin phi, sin th); wavevector (kx_inc, ky_inc, -k0 cos th).
    """
    if pol == 0:
        e = (-math.sin(g.phi), math.cos(g.phi), 0.0)
    else:
        e = (math.cos(g.theta) * math.cos(g.phi), math.cos(g.theta) * math.sin(g.phi), math.sin(g.theta))
    zrel = (torch.arange(g.nz, dtype=F64) - g.z_ml) * g.dz
    ph = torch.exp(-1j * g.kz_inc * zrel.to(C128))
    out = torch.zeros(g.shape, dtype=C128)
    for c in range(3):
        out[c] = e[c] * ph[:, None, None]
    return out


def source_b(g: Grid, fill: torch.Tensor, pol: int) -> torch.Tensor:
    """b = k0^2 deps (E_inc + E_ML) with E_ML = R E_inc (Eq. bg_source)."""
    Einc = incident_field(g, pol)
    de = deps_field(g, fill)[None]
    return g.k0 ** 2 * de * (Einc + reflect(g, Einc))


def residual(g: Grid, E: torch.Tensor, fill: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """r = b - A E and its relative norm (Eq. relative_residual)."""
    r = b.to(C128) - apply_A(g, E, fill)
    return r


def rel_residual(g: Grid, E, fill, b) -> float:
    r = residual(g, E, fill, b)
    return float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b.to(C128)))


def upgoing_amplitude(g: Grid, Etot_y_column: torch.Tensor, k: int) -> complex:
    """Helper for slab tests: amplitude of exp(+i kz_inc (z - z_ml)) in a 1-D column at plane k."""
    zrel = (k - g.z_ml) * g.dz
    return complex(Etot_y_column[k] * torch.exp(torch.tensor(-1j * g.kz_inc * zrel)))


# --------------------------------------------------------------------------- layered-background preconditioner
# Not in the paper: the right preconditioner P = A0^-1 with A0 the operator A whose contrast is
# replaced, on every z-plane, by its lateral mean.  A0 couples no lateral Bloch modes.

def lateral_mean_fill(fill: torch.Tensor) -> torch.Tensor:
    """The fill averaged over every z-plane and broadcast back to (nz, ny, nx)."""
    return fill.to(F64).mean(dim=(1, 2), keepdim=True).expand_as(fill).contiguous()


def layered_blocks(g: Grid, fill: torch.Tensor) -> torch.Tensor:
    """Per-mode matrices of A0, shape (ny, nx, 3 nz, 3 nz), index c * nz + z (c = x, y, z).

    Column (c, z') is A0 applied to a unit source at component c, plane z' and the lateral
    origin: the lateral DFT of that source is 1 in every mode, so the DFT of the output is
    column (c, z') of every mode's matrix at once.
    """
    fbar = lateral_mean_fill(fill)
    n = 3 * g.nz
    mats = torch.zeros(g.ny, g.nx, n, n, dtype=C128)
    for c in range(3):
        for z in range(g.nz):
            E = torch.zeros(g.shape, dtype=C128)
            E[c, z, 0, 0] = 1.0
            Yh = _fft2(apply_A(g, E, fbar))                      # (3, nz, ny, nx)
            mats[:, :, :, c * g.nz + z] = Yh.permute(2, 3, 0, 1).reshape(g.ny, g.nx, n)
    return mats


def apply_P_layered(g: Grid, fill: torch.Tensor, X: torch.Tensor, mats: torch.Tensor = None,
                    lu=None) -> torch.Tensor:
    """y = A0^-1 x per lateral mode (real-space fields (3, nz, ny, nx)).

    ``lu``: the (LU, pivots) of torch.linalg.lu_factor(mats), for repeated applications of the
    same blocks (LU with partial pivoting, factored once); otherwise each call solves with ``mats``."""
    n = 3 * g.nz
    Xh = _fft2(X.to(C128)).permute(2, 3, 0, 1).reshape(g.ny, g.nx, n, 1)
    if lu is not None:
        Yh = torch.linalg.lu_solve(lu[0], lu[1], Xh)
    else:
        if mats is None:
            mats = layered_blocks(g, fill)
        Yh = torch.linalg.solve(mats, Xh)
    Yh = Yh.reshape(g.ny, g.nx, 3, g.nz).permute(2, 3, 0, 1)
    return _ifft2(Yh)


# --------------------------------------------------------------------------- meshed layered structures
def layered_cell_contrast(g: Grid, layers, z_top: float, eps_below: complex) -> torch.Tensor:
    """Cell-averaged eps - 1 of a layer stack meshed on the planes: layers = [(eps, thickness), ...]
    listed top to bottom, the top face at height z_top (nm, plane k at k dz), eps_below under the
    last layer (down into the bottom PML), vacuum above.  Cell k covers [k dz - dz/2, k dz + dz/2]."""
    bounds = [(float("inf"), z_top, 1.0 + 0j)]
    z = z_top
    for eps, d in layers:
        bounds.append((z, z - d, complex(eps)))
        z -= d
    bounds.append((z, -float("inf"), complex(eps_below)))
    c = torch.zeros(g.nz, dtype=C128)
    for k in range(g.nz):
        lo, hi = k * g.dz - 0.5 * g.dz, k * g.dz + 0.5 * g.dz
        acc = 0j
        for top, bot, eps in bounds:
            ov = max(0.0, min(hi, top) - max(lo, bot))
            acc += ov * (eps - 1.0)
        c[k] = acc / g.dz
    return c


def specular_reflection(g: Grid, E: torch.Tensor, z_obs: int, z_top: float, pol: int) -> complex:
    """Reflection coefficient of the tangential field at the stack top from the scattered field in
    the vacuum above it: E_s = r E_inc(z_top) exp(i k_z (z - z_top)) in the incident Bloch mode."""
    Eh = _fft2(E.to(C128)) / (g.nx * g.ny)                        # mode (0, 0) = incident Bloch mode
    kz = g.kz_inc
    einc_top = cmath.exp(-1j * kz * (z_top - g.z_ml * g.dz))       # incident phase at the stack top
    if pol == 0:
        e_t = -math.sin(g.phi) * Eh[0, z_obs, 0, 0] + math.cos(g.phi) * Eh[1, z_obs, 0, 0]
        amp = 1.0
    else:
        e_t = math.cos(g.phi) * Eh[0, z_obs, 0, 0] + math.sin(g.phi) * Eh[1, z_obs, 0, 0]
        amp = math.cos(g.theta)                                    # tangential part of the TM field
    return complex(e_t) / (amp * einc_top * cmath.exp(1j * kz * (z_obs * g.dz - z_top)))
