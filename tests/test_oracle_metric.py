"""Pins of the oracle's threshold-contour width metric (Sec. 4, Eq. logistic_sigmoid).

Facts fixed outside the oracle: a triangle-wave intensity with its kinks on samples is linear
between samples, so linear interpolation finds its threshold crossings exactly and the widths
have a closed form; integer shifts of a periodic field move segments but not widths; a field
compared with itself deviates by zero.
"""
import numpy as np
import pytest

from oracle import metric as MT

I_TH = 0.15


def _triangle(n, period, amp, level):
    """I(x) = I_th + amp (tri(x) - level), tri = 1 at x = 0 mod period, -1 at period/2."""
    x = np.arange(n)
    ph = (x % period) / period
    tri = 1.0 - 4.0 * np.minimum(ph, 1.0 - ph)
    return (I_TH + amp * (tri - level)).astype(np.float32)


def _field(I2):
    ny, nx = I2.shape
    E = np.zeros((3, 2, ny, nx), dtype=np.complex64)
    E[1, 1] = np.sqrt(np.maximum(I2, 0.0)).astype(np.float32)
    return E


@pytest.mark.parametrize("period,level", [(16, 0.3), (32, -0.25), (8, 0.5)])
def test_triangle_wave_widths_are_exact(period, level):
    n = 64
    I = _triangle(n, period, 0.1, level)
    segs = MT.line_segments(I, I_TH)
    # tri > level over |x| < (1 - level) period / 4 around each peak
    w = (1.0 - level) * period / 2.0
    assert len(segs) == n // period
    for a, b in segs:
        assert abs((b - a) - w) < 1e-5
        # centred on a peak (multiple of the period), the first one across the wrap
        c = 0.5 * (a + b) % n
        assert min(c % period, period - c % period) < 1e-5


def test_integer_shift_moves_segments_not_widths():
    rng = np.random.default_rng(3)
    I2 = (0.15 + 0.1 * rng.standard_normal((32, 48))).astype(np.float32)
    E = _field(I2)
    E2 = np.roll(E, shift=(5, -7), axis=(2, 3))
    w1 = sorted(round(b - a, 5) for line in MT.widths(E, 1, I_TH, 100) for a, b in line)
    w2 = sorted(round(b - a, 5) for line in MT.widths(E2, 1, I_TH, 100) for a, b in line)
    assert w1 == w2


def test_self_deviation_is_zero_and_a_narrower_feature_is_measured():
    ny, nx = 16, 64
    base = np.tile(_triangle(nx, 32, 0.1, 0.3), (ny, 1))
    d0 = MT.deviation(_field(base), _field(base), 1, I_TH, 100)
    # rows cross two features each; columns are constant along y (all above or all below): none
    assert d0["mean"] == 0.0 and d0["unresolved"] == 0 and d0["matched"] == 2 * ny
    # raise the level: every segment narrows by (0.5 - 0.3) * 32 / 2 = 3.2 px -> 6.4 nm / 4 = 1.6 nm
    narrow = np.tile(_triangle(nx, 32, 0.1, 0.5), (ny, 1))
    d1 = MT.deviation(_field(narrow), _field(base), 1, I_TH, 100, dx=2.0, dy=2.0)
    assert d1["matched"] == 2 * ny and abs(d1["mean"] - 1.6) < 1e-5 and d1["frac_above_1nm"] == 1.0
    # no feature at all: every reference segment is unresolved
    d2 = MT.deviation(_field(np.zeros_like(base)), _field(base), 1, I_TH, 100)
    assert d2["matched"] == 0 and d2["unresolved"] == 2 * ny
