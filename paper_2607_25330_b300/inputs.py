"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers and
lays out geometry and material data.  Both the CUDA path and the CPU oracle
receive exactly what these generators return.

What is generated
-----------------
* Problem presets (grid sizes, pixel sizes, angles, PML thickness, absorber
  extent) for the workloads the paper studies (Sec. 3: EUV mask, lambda =
  13.5 nm, TE illumination, 40-pair Mo/Si multilayer below the absorber).
* Binary mask layouts a_bin(x, y) in {0, 1} (Sec. 2.1: the mask geometry is a
  binary material indicator that is extruded through the absorber).  The paper
  trains and tests on LithoBench layouts, which are not available here; seeded
  random Manhattan layouts (unions of axis-aligned rectangles) and line/space
  gratings stand in for them.
* The axial profile of the absorber: the fraction of each z cell
  [z_k - dz/2, z_k + dz/2] that lies inside the absorber slab.
* Multilayer stack data (Mo/Si bilayers, optional capping layer).  The paper
  takes its optical constants from an external reference that is not given;
  typical 13.5 nm values are used.
* Random complex fields and factorised-FNO weights (the network's parameters
  are inputs to both implementations).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Dict, List, Optional

import numpy as np

LAMBDA_NM = 13.5
N_ABSORBER = complex(0.94, 0.04)      # absorber refractive index (workload definition)
N_CAP = complex(0.97, 0.01)           # capping layer refractive index
N_MO = complex(0.921, 0.0064)         # molybdenum at 13.5 nm (typical value)
N_SI = complex(0.999, 0.0018)         # silicon at 13.5 nm (typical value)
D_MO_NM = 2.8
D_SI_NM = 4.2
N_PAIRS = 40
D_CAP_NM = 2.5

TE = 0
TM = 1


def multilayer_stack(cap: bool = False) -> Dict:
    """Mo/Si Bragg reflector below the mask domain, listed top to bottom.

    40 bilayers of 7 nm period (Sec. 3), Si on top of each pair, Si substrate.
    With ``cap`` a capping layer is put on top of the stack (it then belongs to
    the analytic background, not to the meshed domain).
    """
    n: List[complex] = []
    d: List[float] = []
    if cap:
        n.append(N_CAP)
        d.append(D_CAP_NM)
    for _ in range(N_PAIRS):
        n += [N_SI, N_MO]
        d += [D_SI_NM, D_MO_NM]
    return {"n": n, "d": d, "n_sub": N_SI}


def empty_stack(n_sub: complex = 1.0 + 0.0j) -> Dict:
    """No multilayer: a homogeneous half space below z_ml (vacuum by default)."""
    return {"n": [], "d": [], "n_sub": complex(n_sub)}


@dataclass
class Problem:
    """Grid and illumination of one PSFD problem (all lengths in nm)."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    lam: float = LAMBDA_NM
    theta_deg: float = 6.0
    phi_deg: float = 0.0
    pml_planes: int = 2
    pml_R0: float = 1e-6
    pml_backing: float = 0.5         # peak loss sigma_b of the PML's absorbing backing (0: none)
    z_ml: int = 2                    # plane index of the multilayer interface
    abs_intervals: float = 0.0       # absorber thickness in units of dz (starts at z_ml)
    n_abs: complex = N_ABSORBER
    cap: bool = False
    sigma_px: float = 1.0            # lateral Gaussian smoothing width in pixels
    m_min: float = 0.0               # spectral damping: floor
    k_ref: float = 0.0               # spectral damping: cutoff (0 -> k0)
    gamma: float = 1.0               # spectral damping: decay exponent
    damp_eps_rel: float = 1e-12      # spectral damping: regulariser / k0^2
    pols: List[int] = field(default_factory=lambda: [TE])

    @property
    def eps_abs(self) -> complex:
        return complex(self.n_abs) ** 2

    def zprofile(self) -> np.ndarray:
        return absorber_zprofile(self.nz, self.z_ml, self.abs_intervals)

    def stack(self) -> Dict:
        return multilayer_stack(self.cap)

    def to_dict(self) -> Dict:
        return asdict(self)


def default_pml(nz: int) -> int:
    return max(2, nz // 8)


def absorber_zprofile(nz: int, z_ml: int, intervals: float) -> np.ndarray:
    """Fraction of each z cell covered by the absorber slab [z_ml, z_ml + intervals*dz].

    Cell k spans [k - 1/2, k + 1/2] in units of dz, so a slab whose faces sit on
    grid planes gives weight 1/2 to its two face planes and 1 in between.
    """
    w = np.zeros(nz, dtype=np.float64)
    lo, hi = float(z_ml), float(z_ml) + float(intervals)
    for k in range(nz):
        a, b = k - 0.5, k + 0.5
        w[k] = max(0.0, min(b, hi) - max(a, lo))
    return w


def absorber_planes(nz: int, pml: int) -> float:
    """Absorber thickness (in dz intervals) for a 2 nm axial grid.

    60 nm (30 intervals) where it fits with room to spare below the top PML,
    otherwise 60 % of the physical planes.
    """
    phys = nz - 2 * pml
    if phys >= 30 + 4:
        return 30.0
    return float(round(0.6 * phys))


# ---------------------------------------------------------------- presets

def preset(name: str) -> Problem:
    """Named workloads (grid, pixels, angle, PML, absorber extent)."""
    if name == "line_space_32x32x16":
        # 32x32 lateral at 2 nm, 16 planes; the absorber fills the physical planes.
        return Problem(nx=32, ny=32, nz=16, dx=2.0, dy=2.0, dz=3.75, theta_deg=6.0,
                       pml_planes=2, z_ml=2, abs_intervals=11.0, cap=False, pols=[TE])
    if name == "manhattan_128x128x64":
        return Problem(nx=128, ny=128, nz=64, dx=2.0, dy=2.0, dz=2.0, theta_deg=6.0,
                       pml_planes=8, z_ml=8, abs_intervals=30.0, cap=True, pols=[TE, TM])
    if name == "fno_train_128x128x48":
        return Problem(nx=128, ny=128, nz=48, dx=2.0, dy=2.0, dz=2.0, theta_deg=6.0,
                       pml_planes=6, z_ml=6, abs_intervals=30.0, cap=True, pols=[TE])
    if name == "fine_512x512x128":
        return Problem(nx=512, ny=512, nz=128, dx=0.5, dy=0.5, dz=2.0, theta_deg=6.0,
                       pml_planes=16, z_ml=16, abs_intervals=30.0, cap=True, pols=[TE, TM])
    if name == "batch_128x128x96":
        # one of the batched workload's (lateral size, depth) pairs: 60 nm absorber, 12 PML planes
        return Problem(nx=128, ny=128, nz=96, dx=2.0, dy=2.0, dz=2.0, theta_deg=6.0,
                       pml_planes=12, z_ml=12, abs_intervals=30.0, cap=True, pols=[TE, TM])
    if name == "fno_coarse_128x128x128":
        # coarse grid of the fine-discretisation warm start: the 512 case's box and axial planes
        # (2 nm, a third of the 13.5 nm wavelength) with 4x coarser lateral pixels
        return Problem(nx=128, ny=128, nz=128, dx=2.0, dy=2.0, dz=2.0, theta_deg=6.0,
                       pml_planes=16, z_ml=16, abs_intervals=30.0, cap=True, pols=[TE, TM])
    if name == "fno_coarse_128x128x32":
        # coarse grid of the fine-discretisation warm start (same physical box as the 512 case)
        return Problem(nx=128, ny=128, nz=32, dx=2.0, dy=2.0, dz=8.0, theta_deg=6.0,
                       pml_planes=4, z_ml=4, abs_intervals=7.5, cap=True, pols=[TE, TM])
    raise KeyError(name)


def batch_presets() -> List[Problem]:
    """64 masks of uneven lateral size and depth: 4 per (lateral size, Nz) pair.

    Each mask is solved at 3 angles x 2 polarisations; the angle is a property of
    the operator (Bloch shift), so one Problem is returned per (mask, angle).
    """
    out = []
    for n in (64, 96, 128, 256):
        for nz in (32, 48, 64, 96):
            pml = default_pml(nz)
            for _m in range(4):
                for ang in (4.0, 6.0, 8.0):
                    out.append(Problem(nx=n, ny=n, nz=nz, dx=2.0, dy=2.0, dz=2.0,
                                       theta_deg=ang, pml_planes=pml, z_ml=pml,
                                       abs_intervals=absorber_planes(nz, pml), cap=True,
                                       pols=[TE, TM]))
    return out


# ---------------------------------------------------------------- masks

def manhattan_mask(ny: int, nx: int, rng: np.random.Generator, nrect=(4, 24),
                   edge=(4, 40)) -> np.ndarray:
    """Union of K ~ U{nrect} axis-aligned rectangles with edges ~ U{edge} pixels.

    Lower-left corners are uniform over the grid; rectangles wrap periodically.
    """
    a = np.zeros((ny, nx), dtype=np.uint8)
    k = int(rng.integers(nrect[0], nrect[1] + 1))
    for _ in range(k):
        w = int(rng.integers(edge[0], edge[1] + 1))
        h = int(rng.integers(edge[0], edge[1] + 1))
        x0 = int(rng.integers(0, nx))
        y0 = int(rng.integers(0, ny))
        ys = (y0 + np.arange(min(h, ny))) % ny
        xs = (x0 + np.arange(min(w, nx))) % nx
        a[np.ix_(ys, xs)] = 1
    return a


def line_space_mask(ny: int, nx: int, rng: np.random.Generator, half_pitch_px: int = 8) -> np.ndarray:
    """Vertical lines (constant in y) of width half_pitch with pitch 2*half_pitch, seeded edge offset."""
    off = int(rng.integers(0, 2 * half_pitch_px))
    x = (np.arange(nx) - off) % (2 * half_pitch_px)
    row = (x < half_pitch_px).astype(np.uint8)
    return np.repeat(row[None, :], ny, axis=0)


def mask_for(prob: Problem, seed: int, kind: Optional[str] = None) -> np.ndarray:
    rng = np.random.default_rng(np.random.PCG64(seed))
    if kind is None:
        kind = "line_space" if prob.nx <= 32 else "manhattan"
    if kind == "line_space":
        return line_space_mask(prob.ny, prob.nx, rng)
    if kind == "manhattan_dense":
        s = max(1, prob.nx // 128)
        return manhattan_mask(prob.ny, prob.nx, rng, nrect=(40, 120), edge=(4 * s, 40 * s))
    if kind == "blank":
        return np.zeros((prob.ny, prob.nx), dtype=np.uint8)
    if kind == "full":
        return np.ones((prob.ny, prob.nx), dtype=np.uint8)
    return manhattan_mask(prob.ny, prob.nx, rng)


# ---------------------------------------------------------------- fields

def random_field(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(np.random.PCG64(seed))
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(dtype)


# ---------------------------------------------------------------- FNO weights

@dataclass
class FNOShape:
    dv: int = 32          # Fourier-layer channels
    dh: int = 64          # MLP hidden channels
    layers: int = 4
    mx: int = 32          # retained lateral modes per axis (k in [-mx/2, mx/2-1])
    my: int = 32
    mz: int = 16          # retained axial modes
    dq: int = 128         # projection hidden width
    n_in: int = 4         # a, x, y, z
    n_out: int = 6        # Re/Im of Ex, Ey, Ez


def fno_weights(shape: FNOShape, seed: int, spectral_scale: float = 1.0) -> Dict[str, np.ndarray]:
    """Seed-initialised factorised-FNO parameters (float32).

    Spectral kernels are complex with entries scale*U[0,1)/(dv*dv) per part, the
    pointwise layers use U(-1/sqrt(fan_in), 1/sqrt(fan_in)).
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    S = shape

    def lin(o, i):
        b = 1.0 / math.sqrt(i)
        return rng.uniform(-b, b, size=(o, i)).astype(np.float32), rng.uniform(-b, b, size=(o,)).astype(np.float32)

    w = {}
    w["lift_w"], w["lift_b"] = lin(S.dv, S.n_in)
    sc = spectral_scale / (S.dv * S.dv)
    kxy = sc * (rng.random((S.layers, S.my, S.mx, S.dv, S.dv)) + 1j * rng.random((S.layers, S.my, S.mx, S.dv, S.dv)))
    kz = sc * (rng.random((S.layers, S.mz, S.dv, S.dv)) + 1j * rng.random((S.layers, S.mz, S.dv, S.dv)))
    w["kxy"] = kxy.astype(np.complex64)     # [L][my][mx][out][in], modes in centred order k = -m/2 .. m/2-1
    w["kz"] = kz.astype(np.complex64)       # [L][mz][out][in]
    w1, b1, w2, b2 = [], [], [], []
    for _ in range(S.layers):
        a, b = lin(S.dh, S.dv); w1.append(a); b1.append(b)
        a, b = lin(S.dv, S.dh); w2.append(a); b2.append(b)
    w["w1"] = np.stack(w1); w["b1"] = np.stack(b1)
    w["w2"] = np.stack(w2); w["b2"] = np.stack(b2)
    w["q1"], w["qb1"] = lin(S.dq, S.dv)
    w["q2"], w["qb2"] = lin(S.n_out, S.dq)
    return w
