"""Pins of the FP64 oracle's PSFD operator against facts fixed outside the oracle.

Each test names the passage or the mathematics it checks.  None of these
re-types an oracle formula: they use closed forms (plane-wave symbol, Fresnel,
quarter-wave stack, Airy slab, periodised Gaussian), identities (div curl = 0,
curl grad = 0, adjoint identity, unit reflectance under total internal
reflection), an independent transfer-matrix product, or a printed value.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import psfd as O
from oracle import krylov as K
from paper_2607_25330_b300 import inputs as I

C128 = torch.complex128
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(nx=6, ny=4, nz=12, pml=2, theta=6.0, phi=0.0, cap=True, **kw):
    p = I.Problem(nx=nx, ny=ny, nz=nz, dx=2.0, dy=2.5, dz=2.0, theta_deg=theta, phi_deg=phi,
                  pml_planes=pml, z_ml=pml, abs_intervals=min(5.0, nz - 2 * pml - 2), cap=cap, **kw)
    return p


def rand_c(shape, seed):
    return torch.from_numpy(I.random_field(shape, seed))


def rand_fill(p, seed):
    rng = np.random.default_rng(seed)
    a = (rng.random((p.ny, p.nx)) > 0.5).astype(np.uint8)
    return O.fill_fraction(a, p.zprofile(), 1.0)


# ---------------------------------------------------------------- wavenumber grid

def test_representable_angles_match_paper():
    """Sec. 3 (Fig. 1(c,d) discussion): theta_m = arcsin(k_xm / k0) = 0, 5.16, 10.37, 15.66 deg."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "representable_angles.txt")) if l.strip() and not l.startswith("#")]
    lam, Lx = map(float, rows[0])
    nx = 150
    p = I.Problem(nx=nx, ny=1, nz=4, dx=Lx / nx, dy=1.0, dz=1.0, lam=lam, theta_deg=0.0, pml_planes=0, z_ml=0)
    g = O.Grid(p.to_dict(), I.empty_stack())
    for m_str, th_str in rows[1:]:
        m = int(m_str)
        th = math.degrees(math.asin(float(g.kx[m]) / g.k0))
        assert round(th, 2) == float(th_str)


# ---------------------------------------------------------------- curl-curl operator

@pytest.mark.parametrize("mode", [(0, 0, 0), (1, 2, 3), (5, 3, 6), (3, 1, 11)])
def test_curlcurl_plane_wave_symbol(mode):
    """Without PML a grid plane wave is an eigenfunction: (curl curl - k0^2) e = (|k|^2 - k k^T - k0^2) e.

    Closed form of Eq. vector_helmholtz_operator for exp(i k.r); includes the
    Nyquist indices (3 of 6, 2 of 4, 6 of 12) and the Bloch shift.
    """
    p = small_problem(pml=0, theta=7.0, phi=20.0)
    g = O.Grid(p.to_dict(), I.empty_stack())
    mx, my, mz = mode
    k = np.array([float(g.kx[mx]), float(g.ky[my]), float(g.kz[mz])])
    kk = k - np.array([g.kx_inc, g.ky_inc, 0.0])                    # envelope wavenumbers
    x = np.arange(g.nx) * g.dx
    y = np.arange(g.ny) * g.dy
    z = np.arange(g.nz) * g.dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    phase = np.exp(1j * (kk[0] * X + kk[1] * Y + kk[2] * Z))
    e = np.array([0.3 + 0.1j, -0.7 + 0.4j, 0.2 - 0.5j])
    E = torch.from_numpy(e[:, None, None, None] * phase[None])
    fill = torch.zeros(g.nz, g.ny, g.nx, dtype=torch.float64)
    out = O.apply_A(g, E, fill).numpy()
    sym = (k @ k) * e - k * (k @ e) - g.k0 ** 2 * e
    ref = sym[:, None, None, None] * phase[None]
    assert np.max(np.abs(out - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def _div(g, F):
    """Stretched divergence i kx Fx + i ky Fy + D_z Fz in real space (D_z with the PML)."""
    Fh = torch.fft.fft2(F, dim=(-2, -1))
    dz = O._dz(g, Fh[2])
    d = 1j * g.KX * Fh[0] + 1j * g.KY * Fh[1] + dz
    return torch.fft.ifft2(d, dim=(-2, -1))


def _grad(g, phi):
    ph = torch.fft.fft2(phi, dim=(-2, -1))
    return torch.fft.ifft2(torch.stack([1j * g.KX * ph, 1j * g.KY * ph, O._dz(g, ph)]), dim=(-2, -1))


def test_divergence_of_curlcurl_vanishes_with_pml():
    """div_s (curl_s curl_s E) = 0: all derivative pairs commute (lateral multipliers vs D_z)."""
    p = small_problem()
    g = O.Grid(p.to_dict(), I.empty_stack())
    E = rand_c(g.shape, 1)
    cc = O.curlcurl(g, E)
    d = _div(g, cc)
    assert float(d.abs().max()) < 1e-11 * float(cc.abs().max())


def test_curlcurl_annihilates_gradients_with_pml():
    """curl_s grad_s phi = 0, so A (grad phi) = -k0^2 eps_bg grad phi where deps = 0."""
    p = small_problem()
    g = O.Grid(p.to_dict(), I.empty_stack())
    phi = rand_c((g.nz, g.ny, g.nx), 2)
    G = _grad(g, phi)
    fill = torch.zeros(g.nz, g.ny, g.nx, dtype=torch.float64)
    out = O.apply_A(g, G, fill)
    assert float((out + g.k0 ** 2 * g.eps_bg[None, :, None, None] * G).abs().max()) < 1e-11 * float(G.abs().max())


@pytest.mark.parametrize("npml,backing", [(4, 0.5), (8, 1.0), (2, 0.5), (4, 0.0)])
def test_pml_backing_damps_the_z_constant_lateral_mode(npml, backing):
    """A field constant in z is annihilated by D_z for any stretch s, so for a lateral mode with
    E perpendicular to k_par the vacuum operator reduces to the closed form
    A E = (|k_par|^2 - k0^2 eps_bg(z)) E: with no backing its Rayleigh quotient is real (an
    undamped mode whose eigenvalue |k_par|^2 - k0^2 vanishes at grazing); the backing adds
    -i k0^2 sigma_b ((nb - j) / nb)^2 on the j-th of the outermost nb = max(1, npml / 4) planes of
    each end, and nothing elsewhere."""
    nz = 4 * npml + 8
    p = I.Problem(nx=6, ny=4, nz=nz, dx=2.0, dy=2.5, dz=2.0, theta_deg=7.0, pml_planes=npml, z_ml=npml,
                  abs_intervals=2.0, pml_backing=backing)
    g = O.Grid(p.to_dict(), I.empty_stack())
    mx, my = 2, 1
    kx, ky = float(g.kx[mx]), float(g.ky[my])
    kk = (kx - g.kx_inc, ky - g.ky_inc)
    x = np.arange(g.nx) * g.dx
    y = np.arange(g.ny) * g.dy
    Y, X = np.meshgrid(y, x, indexing="ij")
    phase = np.exp(1j * (kk[0] * X + kk[1] * Y))
    s_hat = np.array([-ky, kx, 0.0]) / math.hypot(kx, ky)
    E = torch.from_numpy(s_hat[:, None, None, None] * np.broadcast_to(phase, (g.nz, g.ny, g.nx))[None])
    fill = torch.zeros(g.nz, g.ny, g.nx, dtype=torch.float64)
    out = O.apply_A(g, E, fill)
    nb = max(1, npml // 4) if backing > 0 else 0
    sig = np.zeros(nz)
    for j in range(nb):
        sig[j] = sig[nz - 1 - j] = backing * ((nb - j) / nb) ** 2
    lam = (kx ** 2 + ky ** 2) - g.k0 ** 2 * (1.0 + 1j * sig)
    ref = torch.from_numpy(lam)[None, :, None, None] * E
    assert float((out - ref).abs().max()) < 1e-11 * g.k0 ** 2
    rq = complex(torch.vdot(E.flatten(), out.flatten()) / torch.vdot(E.flatten(), E.flatten()))
    assert abs(rq.imag + g.k0 ** 2 * sig.sum() / nz) < 1e-12 * g.k0 ** 2
    assert (sig.sum() > 0) == (backing > 0)


def test_pml_profile_vanishes_in_the_physical_region():
    p = small_problem(nz=20, pml=4)
    g = O.Grid(p.to_dict(), I.empty_stack())
    assert torch.all(g.sigma[4:16] == 0)
    assert torch.all(g.sigma[:4] > 0) and torch.all(g.sigma[16:] > 0)
    # reflection of the profile: sigma is symmetric about the box edge
    assert torch.allclose(g.sigma[:4].flip(0), g.sigma[16:])


# ---------------------------------------------------------------- reflection coefficients

def _kp2(kpar):
    return torch.tensor([[kpar ** 2]], dtype=torch.float64)


@pytest.mark.parametrize("theta", [0.0, 6.0, 30.0, 70.0])
@pytest.mark.parametrize("n2", [1.5, 0.9 + 0.05j, 2.0 + 0.3j])
def test_single_interface_is_fresnel(theta, n2):
    """One interface: Fresnel r_s and the tangential-E ratio of the p wave."""
    k0 = 2 * math.pi / 13.5
    kp = k0 * math.sin(math.radians(theta))
    st = {"n": [], "d": [], "n_sub": n2}
    rs = O.reflection_coefficient(_kp2(kp), st, k0, "s").item()
    rp = O.reflection_coefficient(_kp2(kp), st, k0, "p").item()
    c1 = math.cos(math.radians(theta))
    n2 = complex(n2)
    c2 = np.sqrt(1 - (math.sin(math.radians(theta)) / n2) ** 2 + 0j)
    if c2.imag < 0:
        c2 = -c2
    rs_ref = (c1 - n2 * c2) / (c1 + n2 * c2)
    # tangential-E ratio: (n2 cos1 - cos2 ... ) written through impedances of the p wave
    rp_ref = (n2 * c1 - c2) / (n2 * c1 + c2) * (-1)
    assert abs(rs - rs_ref) < 1e-13
    assert abs(rp - rp_ref) < 1e-13


@pytest.mark.parametrize("npairs", [1, 5, 12])
def test_quarter_wave_stack_closed_form(npairs):
    """Lossless (HL)^N quarter-wave stack at its design wavelength, normal incidence:
    input admittance Y = (nH/nL)^(2N) n_s, r = (1 - Y)/(1 + Y)."""
    lam = 13.5
    k0 = 2 * math.pi / lam
    nH, nL, ns = 1.7, 1.2, 1.45
    st = {"n": [nH, nL] * npairs, "d": [lam / (4 * nH), lam / (4 * nL)] * npairs, "n_sub": ns}
    Y = (nH / nL) ** (2 * npairs) * ns
    ref = (1 - Y) / (1 + Y)
    for pol in "sp":
        r = O.reflection_coefficient(_kp2(0.0), st, k0, pol).item()
        assert abs(r - ref) < 1e-12


def test_total_internal_reflection_has_unit_modulus():
    """Lossless layers over a substrate in which the mode is evanescent: |r| = 1 (energy conservation)."""
    k0 = 2 * math.pi / 13.5
    # propagating in vacuum (kp < k0) and in the layers, evanescent in the n = 0.5 substrate
    st = {"n": [1.3, 1.1, 1.6], "d": [3.0, 5.0, 2.0], "n_sub": 0.5}
    kp = 0.8 * k0
    for pol in "sp":
        r = O.reflection_coefficient(_kp2(kp), st, k0, pol).item()
        assert abs(abs(r) - 1.0) < 1e-13


def test_zero_thickness_layer_is_a_no_op():
    k0 = 2 * math.pi / 13.5
    st = I.multilayer_stack(cap=True)
    st2 = {"n": [3.0 + 1j] + st["n"], "d": [0.0] + st["d"], "n_sub": st["n_sub"]}
    for kp in (0.0, 0.3 * k0, 1.7 * k0):
        for pol in "sp":
            a = O.reflection_coefficient(_kp2(kp), st, k0, pol).item()
            b = O.reflection_coefficient(_kp2(kp), st2, k0, pol).item()
            assert abs(a - b) < 1e-13


def characteristic_matrix_r(kpar, stack, k0, pol):
    """Independent transfer-matrix product of the tangential fields (E, H) layer by layer."""
    def kz(e):
        r = np.sqrt(complex(k0 * k0 * e - kpar * kpar))
        return -r if r.imag < 0 else r

    def q(e):
        return kz(e) if pol == "s" else kz(e) / e

    P = np.eye(2, dtype=complex)
    for n, t in zip(stack["n"], stack["d"]):
        e = complex(n) ** 2
        dl = kz(e) * t
        M = np.array([[np.cos(dl), 1j * np.sin(dl) / q(e)], [1j * q(e) * np.sin(dl), np.cos(dl)]])
        P = M @ P
    qs, q0 = q(complex(stack["n_sub"]) ** 2), q(1.0)
    a = P[1, 0] - qs * P[0, 0]
    c = q0 * (P[1, 1] - qs * P[0, 1])
    r = (a + c) / (c - a)              # ratio of the continuous field (E_y for s, H_y for p)
    return r if pol == "s" else -r     # p: tangential E flips sign relative to H_y


@pytest.mark.parametrize("theta", [0.0, 4.0, 8.0, 20.0])
@pytest.mark.parametrize("cap", [False, True])
def test_multilayer_matches_transfer_matrix_product(theta, cap):
    """Mo/Si stack (40 pairs, Sec. 3) by the Airy recursion vs an explicit 2x2 matrix product."""
    k0 = 2 * math.pi / 13.5
    st = I.multilayer_stack(cap)
    kp = k0 * math.sin(math.radians(theta))
    for pol in "sp":
        a = O.reflection_coefficient(_kp2(kp), st, k0, pol).item()
        b = characteristic_matrix_r(kp, st, k0, pol)
        assert abs(a - b) < 1e-12


def test_multilayer_reflectance_is_euv_like():
    """Sanity of the stack data: peak reflectance of order 0.7 near normal incidence."""
    k0 = 2 * math.pi / 13.5
    r = O.reflection_coefficient(_kp2(0.0), I.multilayer_stack(False), k0, "s").item()
    assert 0.6 < abs(r) ** 2 < 0.8


def test_normal_incidence_s_equals_p():
    k0 = 2 * math.pi / 13.5
    st = I.multilayer_stack(True)
    a = O.reflection_coefficient(_kp2(0.0), st, k0, "s").item()
    b = O.reflection_coefficient(_kp2(0.0), st, k0, "p").item()
    assert abs(a - b) < 1e-14


# ---------------------------------------------------------------- background decomposition

def test_blank_mask_gives_zero_source_and_zero_field():
    """Blank mask: deps = 0, so b = 0 and the scattered field is exactly 0 (Sec. 2.2)."""
    p = small_problem()
    g = O.Grid(p.to_dict(), I.multilayer_stack(True))
    fill = O.fill_fraction(np.zeros((p.ny, p.nx), np.uint8), p.zprofile(), 1.0)
    for pol in (0, 1):
        b = O.source_b(g, fill, pol)
        assert float(b.abs().max()) == 0.0
        res = K.solve(lambda E: O.apply_A(g, E, fill), None, b)
        assert float(res["E"].abs().max()) == 0.0 and res["iters"] == 0


def test_incident_field_is_a_transverse_unit_plane_wave():
    p = small_problem(theta=8.0, phi=30.0)
    g = O.Grid(p.to_dict(), I.empty_stack())
    k = np.array([g.kx_inc, g.ky_inc, -g.kz_inc])
    for pol in (0, 1):
        e = O.incident_field(g, pol)[:, g.z_ml, 0, 0].numpy()
        assert abs(np.linalg.norm(e) - 1) < 1e-14
        assert abs(k @ e) < 1e-14


def test_reflected_field_is_upgoing_and_divergence_free():
    """Per lateral mode the reflected vector satisfies k_par . E_par + k_z E_z = 0 and has profile exp(i k_z z)."""
    p = small_problem(theta=8.0, phi=25.0)
    g = O.Grid(p.to_dict(), I.multilayer_stack(True))
    E = rand_c(g.shape, 3)
    R = O.reflect(g, E)
    Rh = torch.fft.fft2(R, dim=(-2, -1))
    v = Rh[:, g.z_ml]
    div = g.KX * v[0] + g.KY * v[1] + g.kz0 * v[2]
    assert float(div.abs().max()) < 1e-12 * float(v.abs().max())
    k = g.z_ml + 3
    ratio = Rh[:, k] / torch.where(v.abs() > 0, v, torch.ones_like(v))
    expect = torch.exp(1j * g.kz0 * 3 * g.dz)
    mask = v.abs() > 1e-8 * float(v.abs().max())
    assert float((ratio - expect[None])[mask].abs().max()) < 1e-12
    assert float(Rh[:, : g.z_ml].abs().max()) == 0.0


def _slab_reflection(dz, h_nm, theta, pol, stack, pml_nm=20.0, vac_nm=20.0):
    """Solve a laterally uniform absorber slab on a 1x1xNz grid (dense LU) and read off the
    specular reflection of the total field above it, referenced at the slab top."""
    npml = int(round(pml_nm / dz))
    nab = h_nm / dz
    nvac = int(round(vac_nm / dz))
    nz = 2 * npml + int(round(nab)) + 1 + nvac
    p = I.Problem(nx=1, ny=1, nz=nz, dx=1.0, dy=1.0, dz=dz, theta_deg=theta, pml_planes=npml,
                  z_ml=npml, abs_intervals=nab)
    g = O.Grid(p.to_dict(), stack)
    fill = O.fill_fraction(np.ones((1, 1), np.uint8), p.zprofile(), 1.0)
    b = O.source_b(g, fill, pol)
    E = K.dense_solve(K.dense_matrix(lambda X: O.apply_A(g, X, fill), g.shape), b)
    Einc = O.incident_field(g, pol)
    comp = 1 if pol == 0 else 0
    up = (O.reflect(g, Einc) + E + O.reflect(g, E))[comp]
    kobs = npml + int(round(nab)) + 1 + nvac // 2
    amp = complex(up[kobs, 0, 0]) * np.exp(-1j * g.kz_inc * (kobs - g.z_ml) * dz)
    amp /= 1.0 if pol == 0 else math.cos(g.theta)     # incident tangential amplitude
    return amp * np.exp(2j * g.kz_inc * h_nm), g


def _airy(theta, n, h, lam, pol):
    """Closed-form reflection of a homogeneous slab in vacuum (tangential-E ratio)."""
    k0 = 2 * math.pi / lam
    c0 = math.cos(math.radians(theta))
    s0 = math.sin(math.radians(theta))
    c1 = np.sqrt(1 - (s0 / n) ** 2 + 0j)
    if c1.imag < 0:
        c1 = -c1
    if pol == 0:
        r01 = (c0 - n * c1) / (c0 + n * c1)
    else:
        r01 = -(n * c0 - c1) / (n * c0 + c1)
    e = np.exp(2j * k0 * n * c1 * h)
    return r01 * (1 - e) / (1 - r01 ** 2 * e)


@pytest.mark.parametrize("pol", [0, 1])
def test_absorber_slab_in_vacuum_matches_airy_formula(pol):
    """Homogeneous absorber (n = 0.94+0.04i, 20 nm) with no multilayer: the 3-D operator
    reduces to 1-D and must reproduce the Airy slab reflection, converging under z refinement."""
    errs = []
    for dz in (1.0, 0.5):
        r, g = _slab_reflection(dz, 20.0, 6.0, pol, I.empty_stack())
        errs.append(abs(r - _airy(6.0, I.N_ABSORBER, 20.0, g.lam, pol)))
    assert errs[1] < 1e-3
    assert errs[1] < errs[0] / 2.5


@pytest.mark.parametrize("pol", [0, 1])
def test_absorber_slab_on_multilayer_matches_transfer_matrix(pol):
    """The background decomposition with R in the operator reproduces the reflection of
    [absorber slab | cap | 40 x Mo/Si] (Sec. 2.2; Fig. 1 accuracy claim), second order in dz."""
    st = I.multilayer_stack(True)
    st2 = {"n": [I.N_ABSORBER] + st["n"], "d": [20.0] + st["d"], "n_sub": st["n_sub"]}
    errs = []
    for dz in (1.0, 0.5):
        r, g = _slab_reflection(dz, 20.0, 6.0, pol, st)
        ref = characteristic_matrix_r(g.kx_inc, st2, g.k0, "s" if pol == 0 else "p")
        errs.append(abs(r - ref))
    assert errs[1] < 1e-3
    assert errs[1] < errs[0] / 3.0


# ---------------------------------------------------------------- adjoint, preconditioner

def test_adjoint_identity():
    """<A x, y> = <x, A^H y> with PML, multilayer reflection and a random contrast."""
    p = small_problem(theta=8.0, phi=15.0)
    g = O.Grid(p.to_dict(), I.multilayer_stack(True))
    fill = rand_fill(p, 4)
    x, y = rand_c(g.shape, 5), rand_c(g.shape, 6)
    lhs = torch.vdot(O.apply_A(g, x, fill).flatten(), y.flatten())
    rhs = torch.vdot(x.flatten(), O.apply_AH(g, y, fill).flatten())
    assert abs(complex(lhs - rhs)) < 1e-12 * abs(complex(lhs))
    lhs = torch.vdot(O.reflect(g, x).flatten(), y.flatten())
    rhs = torch.vdot(x.flatten(), O.reflect_adjoint(g, y).flatten())
    assert abs(complex(lhs - rhs)) < 1e-12 * abs(complex(lhs))


def test_adjoint_is_dense_conjugate_transpose():
    p = small_problem(nx=2, ny=2, nz=8, pml=2, theta=6.0)
    g = O.Grid(p.to_dict(), I.multilayer_stack(True))
    fill = rand_fill(p, 7)
    A = K.dense_matrix(lambda X: O.apply_A(g, X, fill), g.shape)
    AH = K.dense_matrix(lambda X: O.apply_AH(g, X, fill), g.shape)
    assert float((A.conj().T - AH).abs().max()) < 1e-12 * float(A.abs().max())


def test_damping_reduces_to_isotropic_baseline():
    """Eq. spectral_damping_mask with m_min = 0, gamma = 1, eps -> 0, k_ref = k_bg gives min(1, k_bg^2/k^2)."""
    p = small_problem(m_min=0.0, gamma=1.0, k_ref=0.0, damp_eps_rel=0.0)
    g = O.Grid(p.to_dict(), I.empty_stack())
    m = O.damping_multiplier(g)
    k2 = g.kz[:, None, None] ** 2 + g.KY[None] ** 2 + g.KX[None] ** 2
    ref = torch.clamp(g.k0 ** 2 / k2, max=1.0)
    assert torch.allclose(m, ref, rtol=1e-14, atol=0)


def test_damping_floor_and_exponent():
    p = small_problem(m_min=0.2, gamma=0.5, k_ref=0.3, damp_eps_rel=1e-3)
    g = O.Grid(p.to_dict(), I.empty_stack())
    m = O.damping_multiplier(g)
    k2 = (g.kz[:, None, None] ** 2 + g.KY[None] ** 2 + g.KX[None] ** 2).numpy()
    eps = 1e-3 * g.k0 ** 2
    ref = np.where(np.sqrt(k2) <= 0.3, 1.0, 0.2 + 0.8 * np.sqrt(0.09 / (k2 + eps)))
    assert np.allclose(m.numpy(), ref, rtol=1e-14, atol=0)
    assert float(m.min()) >= 0.2 and float(m.max()) <= 1.0


def test_preconditioner_acts_on_plane_waves_and_is_hermitian():
    """Eq. spectral_damping_action: M e^{ik.r} = m(k) e^{ik.r}; M is Hermitian positive definite."""
    p = small_problem(m_min=0.1, gamma=1.0)
    g = O.Grid(p.to_dict(), I.empty_stack())
    m = O.damping_multiplier(g)
    mz, my, mx = 5, 1, 4
    x = torch.arange(g.nx, dtype=torch.float64) * g.dx
    y = torch.arange(g.ny, dtype=torch.float64) * g.dy
    z = torch.arange(g.nz, dtype=torch.float64) * g.dz
    Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
    kk = (float(g.kx[mx]) - g.kx_inc, float(g.ky[my]) - g.ky_inc, float(g.kz[mz]))
    pw = torch.exp(1j * (kk[0] * X + kk[1] * Y + kk[2] * Z))
    E = torch.stack([pw, 2 * pw, -pw])
    out = O.apply_M(g, E)
    assert float((out - m[mz, my, mx] * E).abs().max()) < 1e-13
    a, b = rand_c(g.shape, 8), rand_c(g.shape, 9)
    lhs = torch.vdot(O.apply_M(g, a).flatten(), b.flatten())
    rhs = torch.vdot(a.flatten(), O.apply_M(g, b).flatten())
    assert abs(complex(lhs - rhs)) < 1e-12 * abs(complex(lhs))
    assert float(torch.vdot(a.flatten(), O.apply_M(g, a).flatten()).real) > 0


# ---------------------------------------------------------------- geometry

def test_gaussian_smoothing_of_a_pixel_is_the_periodised_gaussian():
    """Sec. 2.1 smoothing: spectral exp(-sigma^2 kappa^2 / 2) of a unit pixel equals the sampled,
    periodised, unit-mass Gaussian (Poisson summation; spectral truncation error exp(-sigma^2 pi^2/2))."""
    ny, nx, s = 24, 32, 3.0
    a = torch.zeros(ny, nx)
    a[5, 7] = 1.0
    out = O.gaussian_smooth(a, s).numpy()

    def per(n, c):
        x = np.arange(n)
        return sum(np.exp(-((x - c + j * n) ** 2) / (2 * s * s)) for j in range(-3, 4)) / (math.sqrt(2 * math.pi) * s)

    ref = per(ny, 5)[:, None] * per(nx, 7)[None, :]
    assert np.max(np.abs(out - ref)) < 1e-15
    assert abs(out.sum() - 1.0) < 1e-13


def test_fill_is_extruded_and_bounded():
    p = I.preset("line_space_32x32x16")
    a = I.mask_for(p, 3)
    f = O.fill_fraction(a, p.zprofile(), p.sigma_px)
    assert float(f.min()) > -1e-3 and float(f.max()) < 1 + 1e-3
    assert float(f[: p.z_ml].abs().max()) == 0.0
    assert torch.allclose(f[p.z_ml + 1], f[p.z_ml + 2])
    assert torch.allclose(f[p.z_ml], 0.5 * f[p.z_ml + 1])
