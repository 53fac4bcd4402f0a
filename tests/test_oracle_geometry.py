"""Pins of the oracle's overlap geometry (section 2.1 step 1, section 3.1)
against brute-force per-pixel coverage and closed forms."""
import numpy as np
import pytest

from oracle import geometry as geo
from synth import make_rig, rig_for_config


def _T(tx, ty):
    return np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])


def test_integer_translation_band_closed_form():
    # Camera a at x 0..199, camera b shifted by 120: shared columns 120..199.
    g = geo.Geometry([_T(0, 0), _T(120, 0)], [200, 200], [100, 100], 320, 100)
    assert g.bands == [(120, 200, 0, 100)]
    assert g.rects == [((120, 200, 0, 100), (0, 80, 0, 100))]
    assert g.pairs == [(0, 1)]          # reference = camera 1 (n // 2)
    assert g.own_columns(0) == (0, 120)
    assert g.own_columns(1) == (200, 320)


def test_vertical_offset_band_rows():
    g = geo.Geometry([_T(0, 5), _T(150, -3)], [200, 200], [100, 100], 360, 110)
    x0, x1, y0, y1 = g.bands[0]
    assert (x0, x1) == (150, 200)
    # a covers rows 5..104, b covers -3..96 -> common 5..96
    assert (y0, y1) == (5, 97)
    assert g.rects[0] == ((150, 200, 0, 92), (0, 50, 8, 100))


def test_colour_pair_directions():
    assert geo.colour_pairs(4, 2) == [(0, 1), (1, 2), (3, 2)]
    assert geo.colour_pairs(2, 1) == [(0, 1)]
    assert geo.colour_pairs(3, 0) == [(1, 0), (2, 1)]
    assert geo.colour_pairs(8, 4) == [(0, 1), (1, 2), (2, 3), (3, 4), (5, 4), (6, 5), (7, 6)]


def _cov(g, k, xs, ys):
    c, _, _, _ = geo.coverage(g.Hinv[k], g.w[k], g.h[k], xs.astype(float), ys.astype(float))
    return c


@pytest.mark.parametrize("name,seed", [("2x640x360", 0), ("2x640x360", 3), ("4x1920x1080", 1),
                                       ("3x1920x1080", 2)])
def test_band_is_covered_and_maximal(name, seed):
    rig, _ = rig_for_config(name, seed=seed)
    g = geo.Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h)
    for p, (x0, x1, y0, y1) in enumerate(g.bands):
        assert x1 - x0 >= 2 and y1 - y0 >= 2
        ys, xs = np.mgrid[y0:y1, x0:x1]
        xs, ys = xs.ravel(), ys.ravel()
        assert _cov(g, p, xs, ys).all(), "band pixel not covered by the left camera"
        assert _cov(g, p + 1, xs, ys).all(), "band pixel not covered by the right camera"
        # Not much smaller than the doubly covered region: the band holds most
        # of the pixels that both cameras see (the corner-based bounds lose only
        # the slivers cut off by the cameras' rotation).
        lo = max(0, x0 - 200)
        hi = min(g.pano_w, x1 + 200)
        ys2, xs2 = np.mgrid[0:g.pano_h, lo:hi]
        xs2, ys2 = xs2.ravel(), ys2.ravel()
        both = (_cov(g, p, xs2, ys2) & _cov(g, p + 1, xs2, ys2)).sum()
        assert (x1 - x0) * (y1 - y0) > 0.75 * both
    # Bands are ordered and disjoint.
    for p in range(len(g.bands) - 1):
        assert g.bands[p][1] <= g.bands[p + 1][0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_source_rect_maps_into_band(seed):
    rig, _ = rig_for_config("2x640x360", seed=seed)
    g = geo.Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h)
    x0, x1, y0, y1 = g.bands[0]
    for side, cam in ((0, 0), (1, 1)):
        rx0, rx1, ry0, ry1 = g.rects[0][side]
        assert 0 <= rx0 < rx1 <= g.w[cam] and 0 <= ry0 < ry1 <= g.h[cam]
        v, u = np.mgrid[ry0:ry1, rx0:rx1]
        X, Y, _ = geo.project(g.H[cam], u.ravel().astype(float), v.ravel().astype(float))
        eps = 1e-6
        assert (X >= x0 - eps).all() and (X <= x1 - 1 + eps).all()
        assert (Y >= y0 - eps).all() and (Y <= y1 - 1 + eps).all()
        # and the rect is not trivially small: it holds most of the band's area
        assert (rx1 - rx0) * (ry1 - ry0) > 0.75 * (x1 - x0) * (y1 - y0)


def test_inverse_roundtrip_and_coverage_corners():
    rig = make_rig([300, 300], [200, 200], overlap=(0.3, 0.3), rot_deg=3.0, seed=5)
    g = geo.Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h)
    for k in range(2):
        assert np.allclose(g.Hinv[k] @ g.H[k], np.eye(3), atol=1e-12)
        corners = geo.camera_corners(g.H[k], g.w[k], g.h[k])
        sx, sy, _ = geo.project(g.Hinv[k], corners[:, 0], corners[:, 1])
        assert np.allclose(sx, [0, 299, 299, 0]) and np.allclose(sy, [0, 0, 199, 199])


def test_snap_rounding():
    assert geo.ceil_snap(4.0000000000001) == 4
    assert geo.ceil_snap(4.001) == 5
    assert geo.floor_snap(3.9999999999999) == 4
    assert geo.floor_snap(3.999) == 3
