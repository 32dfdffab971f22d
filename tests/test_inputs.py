"""Seeded input generators: determinism and the stated recipe (no method arithmetic here)."""
import numpy as np

from paper_2607_25330_b300 import inputs as I


def test_generators_are_deterministic():
    p = I.preset("manhattan_128x128x64")
    a1, a2 = I.mask_for(p, 11), I.mask_for(p, 11)
    assert np.array_equal(a1, a2) and a1.dtype == np.uint8
    assert not np.array_equal(a1, I.mask_for(p, 12))
    assert np.array_equal(I.random_field((3, 4), 5), I.random_field((3, 4), 5))


def test_zprofile_is_the_cell_overlap():
    w = I.absorber_zprofile(16, 2, 11.0)
    assert w[2] == 0.5 and w[13] == 0.5 and np.all(w[3:13] == 1.0)
    assert abs(w.sum() - 11.0) < 1e-15 and w[:2].sum() == 0 and w[14:].sum() == 0


def test_line_space_has_the_stated_half_pitch():
    p = I.preset("line_space_32x32x16")
    a = I.mask_for(p, 3)
    assert np.all(a == a[0:1])                     # lines along y
    assert a[0].sum() == 16                        # two 8-pixel lines in a 32-pixel period


def test_batch_recipe():
    ps = I.batch_presets()
    assert len(ps) == 192                          # 64 masks x 3 angles
    assert sorted({p.nx for p in ps}) == [64, 96, 128, 256]
    assert sorted({p.nz for p in ps}) == [32, 48, 64, 96]
    assert all(p.z_ml + p.abs_intervals < p.nz - p.pml_planes for p in ps)
