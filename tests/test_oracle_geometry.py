"""Pins of the oracle's pupil geometry (Sec. 2.F masks, Sec. 2.E index order)."""
import numpy as np

from oracle import geometry as geo


def test_hand_counted_tiny_masks():
    # n = 4, no obstruction: centres at +-0.5, +-1.5 (units of d); the four corners
    # lie at radius 1.5*sqrt(2) = 2.12 > 2 = D/2, every other centre is inside.
    m = geo.subaperture_mask(4, 0.0)
    expect = np.array([[0, 1, 1, 0], [1, 1, 1, 1], [1, 1, 1, 1], [0, 1, 1, 0]], bool)
    assert (m == expect).all()
    # phase points: corners of valid subapertures -> all but the 4 outer corners
    pm = geo.phase_point_mask(4, 0.0)
    assert pm.sum() == 25 - 4
    assert not pm[0, 0] and not pm[4, 4] and pm[2, 2]


def test_obstruction_removes_centre():
    # n = 4, obstruction 0.5: the central 4 centres sit at radius 0.707 d < 1 d = 0.5 D/2
    m = geo.subaperture_mask(4, 0.5)
    assert m.sum() == 8 and not m[1:3, 1:3].any()


def test_mask_against_float_distance_rule():
    # brute force with floating-point centre radii (away from exact ties)
    for n, eps in [(20, 0.0), (74, 0.28), (16, 0.28), (10, 0.28), (33, 0.1)]:
        D = 1.0
        d = D / n
        c = (np.arange(n) + 0.5 - n / 2) * d
        yy, xx = np.meshgrid(c, c, indexing="ij")
        r = np.hypot(xx, yy)
        brute = (r <= D / 2 + 1e-12) & (r >= eps * D / 2 - 1e-12)
        assert (geo.subaperture_mask(n, eps) == brute).all()


def test_counts_of_the_workload_grids():
    assert geo.subaperture_mask(20, 0.0).sum() == 316
    assert geo.subaperture_mask(74, 0.28).sum() == 3972
    assert geo.phase_point_mask(74, 0.28).sum() == 4160


def test_row_major_order():
    m = geo.subaperture_mask(6, 0.0)
    v = geo.valid_list(m)
    keys = v[:, 0] * 6 + v[:, 1]
    assert (np.diff(keys) > 0).all()
    cen = geo.subaperture_centres(6, 3.0, 0.0)
    assert np.allclose(cen[:, 0], (v[:, 1] + 0.5 - 3) * 0.5)
    assert np.allclose(cen[:, 1], (v[:, 0] + 0.5 - 3) * 0.5)
