"""Pins of the oracle's cylindrical projection (the large-rig panorama
surface) against closed forms, and of the learned mode's window pooling."""
import math

import numpy as np
import pytest

from oracle.geometry import CylCam, CylMap, Geometry
from synth import rig_for_config


def _K(f, cu, cv):
    return np.array([[f, 0.0, cu], [0.0, f, cv], [0.0, 0.0, 1.0]])


def _ry(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def test_forward_camera_closed_form():
    # camera looking down +z (R = I): the panorama row through the centre maps to
    # u = cu + f tan(theta), v = cv; a panorama height h maps to v = cv + f h / cos(theta)
    f, cu, cv = 500.0, 319.5, 179.5
    C = np.linalg.inv(_K(f, cu, cv))          # camera pixel -> ray
    fp, cx, cy = 500.0, 1000.0, 179.5
    m = CylMap(np.linalg.inv(C), fp, cx, cy)
    for th in (-0.5, -0.1, 0.0, 0.3):
        for h in (-0.2, 0.0, 0.15):
            x, y = cx + fp * th, cy + fp * h
            sx, sy, sw = m.point(x, y)
            assert sw > 0
            assert abs(sx - (cu + f * math.tan(th))) < 1e-9
            assert abs(sy - (cv + f * h / math.cos(th))) < 1e-9
            # vectorised map gives the same point
            vx, vy, _ = m.map(np.array([x]), np.array([y]))
            assert abs(vx[0] - sx) < 1e-9 and abs(vy[0] - sy) < 1e-9


def test_yaw_shifts_the_panorama_by_f_psi():
    f, cu, cv = 700.0, 639.5, 359.5
    psi = 0.37
    C0 = np.linalg.inv(_K(f, cu, cv))                    # R = I
    C1 = _ry(psi) @ np.linalg.inv(_K(f, cu, cv))         # the camera turned by psi about the vertical axis
    fp, cx, cy = 650.0, 3000.0, 359.5
    a, b = CylCam(C0, fp, cx, cy), CylCam(C1, fp, cx, cy)
    rng = np.random.default_rng(0)
    for _ in range(50):
        u, v = rng.uniform(0, 1279), rng.uniform(0, 719)
        x0, y0 = a.point(u, v)
        x1, y1 = b.point(u, v)
        assert abs((x1 - x0) - fp * psi) < 1e-9
        assert abs(y1 - y0) < 1e-9


@pytest.mark.parametrize("seed", [0, 3])
def test_maps_are_inverse_of_each_other(seed):
    rig, _ = rig_for_config("4x640x360cyl", seed=seed)
    f, cx, cy = rig.extra["cyl"]
    rng = np.random.default_rng(seed)
    for k in range(rig.n_cams):
        to_pano = CylCam(rig.H[k], f, cx, cy)
        to_cam = CylMap(np.linalg.inv(rig.H[k]), f, cx, cy)
        u = rng.uniform(0, rig.cam_w[k] - 1, 200)
        v = rng.uniform(0, rig.cam_h[k] - 1, 200)
        X, Y, _ = to_pano.map(u, v)
        su, sv, sw = to_cam.map(X, Y)
        assert np.all(sw > 0)
        assert np.max(np.abs(su - u)) < 1e-7 and np.max(np.abs(sv - v)) < 1e-7


def test_cylindrical_band_lies_in_both_cameras_by_brute_force():
    rig, _ = rig_for_config("4x640x360cyl", seed=1)
    g = Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, projection=1, cyl=rig.extra["cyl"])
    for p, (x0, x1, y0, y1) in enumerate(g.bands):
        X, Y = np.meshgrid(np.arange(x0, x1, dtype=np.float64), np.arange(y0, y1, dtype=np.float64))
        for cam in (p, p + 1):
            sx, sy, sw = g.Hinv[cam].map(X, Y)
            assert np.all(sw > 0)
            assert np.all((sx >= 0) & (sx <= rig.cam_w[cam] - 1) & (sy >= 0) & (sy <= rig.cam_h[cam] - 1))
        # one more column on either side is not covered by both cameras in every band row
        for x in (x0 - 1, x1):
            ok = True
            for cam in (p, p + 1):
                sx, sy, sw = g.Hinv[cam].map(np.full(y1 - y0, float(x)), np.arange(y0, y1, dtype=np.float64))
                ok &= bool(np.all((sw > 0) & (sx >= 0) & (sx <= rig.cam_w[cam] - 1)))
            assert not ok


def test_learned_features_of_a_repeated_frame_equal_one_frame():
    """Window pooling: the same frame W times gives the features of one frame
    (scaled histograms do not depend on the pixel count)."""
    from oracle.pipeline import OracleStitcher
    from synth import Scene, render_camera_frames
    rig, seq = rig_for_config("2x640x360", seed=3)
    scene = Scene(rig.pano_w, rig.pano_h, seed=3)
    frames = [f.numpy() for f in render_camera_frames(rig, scene, 0)]
    a = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=3)
    b = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=3)
    a.estimate_color(frames)
    for _ in range(3):
        b.estimate_color(frames)
    assert np.array_equal(a.learned_features(), b.learned_features())
    # and the features are the scaled overlap histograms: each channel sums to 256 (bf16 rounding aside)
    f = a.learned_features()[0]
    for c in range(6):
        assert abs(f[256 * c:256 * (c + 1)].sum() - 256.0) < 2.0
