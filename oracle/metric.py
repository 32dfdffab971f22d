"""Oracle: threshold-contour width metric of the scattered near field (Sec. 4, practical
assessment of scattered-field convergence; Eq. logistic_sigmoid).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Definition followed:
* intensity I = |E_y^scat|^2 on one z-plane (the first plane above the absorber top);
* the contour is S(I) = 0.5 of the logistic map S, i.e. I = I_th (the transition width w of S
  does not move that contour, so it does not enter the widths);
* along a scan line (a row or a column of the periodic grid) the contour crosses between samples
  j and j + 1 when I_j - I_th and I_{j+1} - I_th have opposite signs (a sample equal to I_th
  counts as above); the crossing sits at j + (I_th - I_j) / (I_{j+1} - I_j) (linear interpolation);
* a segment is a run of above-threshold samples bounded by an upward and a downward crossing;
  its width is the distance between them times the pixel size, with the periodic wrap;
* deviation: every reference segment is matched to the segment of the field under test whose
  centre lies inside it (nearest centre if several); delta d = d_ref - d, reported in wafer
  units |delta d| / demag with demag = 4; a reference segment with no match is "unresolved".
Scan lines: m = min(n_lines, n) rows (columns) at positions floor(i * n / m), i < m.
The above/below decisions are taken on I computed in float32 from the complex64 field, the
precision of the GPU path.

Parity pins (tests/test_oracle_metric.py): triangle-wave intensities whose linear interpolation
is exact give the closed-form widths; integer shifts of the field leave widths unchanged; a
segment across the periodic boundary; the deviation of a field from itself is zero.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np


def line_segments(I: np.ndarray, I_th: float) -> List[Tuple[float, float]]:
    """Above-threshold segments (start, end) in sample units along one periodic line; end > start
    (end may exceed n when the segment wraps)."""
    I = np.asarray(I, dtype=np.float32)
    n = I.shape[0]
    above = I >= np.float32(I_th)
    if above.all() or not above.any():
        return []
    ups, downs = [], []
    for j in range(n):
        a0, a1 = above[j], above[(j + 1) % n]
        if a0 == a1:
            continue
        i0, i1 = float(I[j]), float(I[(j + 1) % n])
        x = j + (I_th - i0) / (i1 - i0)
        (ups if a1 else downs).append(x)
    segs = []
    for u in ups:
        # the first downward crossing after u (periodically)
        d = min((d if d > u else d + n) for d in downs)
        segs.append((u, d))
    return sorted(segs)


def scan_lines(I2: np.ndarray, n_lines: int) -> List[np.ndarray]:
    """Rows then columns of a 2-D periodic intensity (ny, nx) at floor(i * n / n_lines)."""
    ny, nx = I2.shape
    my, mx = min(n_lines, ny), min(n_lines, nx)
    rows = [(i * ny) // my for i in range(my)]
    cols = [(i * nx) // mx for i in range(mx)]
    return [I2[r, :] for r in rows] + [I2[:, c] for c in cols]


def intensity(E: np.ndarray, z: int, comp: int = 1) -> np.ndarray:
    """|E_comp(z)|^2 in float32 from a complex64 field (3, nz, ny, nx)."""
    e = np.asarray(E)[comp, z].astype(np.complex64)
    return (e.real.astype(np.float32) ** 2 + e.imag.astype(np.float32) ** 2).astype(np.float32)


def widths(E: np.ndarray, z: int, I_th: float = 0.15, n_lines: int = 100, comp: int = 1,
           pixel: Tuple[float, float] = (1.0, 1.0)) -> List[List[Tuple[float, float]]]:
    """Segments of every scan line (rows first; pixel = (dx, dy) in nm for rows / columns)."""
    lines = scan_lines(intensity(E, z, comp), n_lines)
    return [line_segments(l, I_th) for l in lines]


def deviation(E: np.ndarray, E_ref: np.ndarray, z: int, I_th: float = 0.15, n_lines: int = 100,
              comp: int = 1, dx: float = 2.0, dy: float = 2.0, demag: float = 4.0) -> Dict:
    """Mean / std / max of |d_ref - d| / demag over matched reference segments, unresolved count."""
    I = intensity(E, z, comp)
    Iref = intensity(E_ref, z, comp)
    ny, nx = I.shape
    n_rows = min(n_lines, ny)
    L, Lr = scan_lines(I, n_lines), scan_lines(Iref, n_lines)
    dev, unresolved = [], 0
    for k, (l, lr) in enumerate(zip(L, Lr)):
        n = l.shape[0]
        px = dx if k < n_rows else dy
        segs, refs = line_segments(l, I_th), line_segments(lr, I_th)
        for (a, b) in refs:
            best, bd = None, None
            for (c, d) in segs:
                ctr = 0.5 * (c + d)
                for shift in (-n, 0, n):
                    cc = ctr + shift
                    if a <= cc <= b:
                        dist = abs(cc - 0.5 * (a + b))
                        if bd is None or dist < bd:
                            best, bd = (c, d), dist
            if best is None:
                unresolved += 1
            else:
                dev.append(abs((b - a) - (best[1] - best[0])) * px / demag)
    dev = np.asarray(dev, dtype=np.float64)
    return {"mean": float(dev.mean()) if dev.size else 0.0, "std": float(dev.std()) if dev.size else 0.0,
            "max": float(dev.max()) if dev.size else 0.0, "matched": int(dev.size), "unresolved": unresolved,
            "frac_above_1nm": float((dev > 1.0).mean()) if dev.size else 0.0}
