"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/stitch.h declares, computes the same overlap
geometry as the oracle, and rejects invalid configurations before touching
the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.geometry import Geometry
from paper_2308_09209_b300 import build as _build
from paper_2308_09209_b300 import stitch as S
from synth import rig_for_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "stitch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stitch_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert "stitch_init" in names and "stitch_frame" in names and len(names) >= 15
    L = ctypes.CDLL(S.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("name", ["2x640x360", "4x1920x1080", "6x1920x1080", "2x1280x720",
                                  "3x1920x1080", "4x3840x2160"])
@pytest.mark.parametrize("seed", [0, 1, 4])
def test_geometry_matches_oracle(name, seed):
    rig, _ = rig_for_config(name, seed=seed)
    cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h)
    bands, rects = S.stitch_geometry(cfg)
    g = Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h)
    assert [tuple(b) for b in bands.tolist()] == g.bands
    assert [tuple(map(tuple, r)) for r in rects.tolist()] == g.rects


def _cfg_of(rig, **kw):
    ex = rig.extra or {}
    return S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, projection=ex.get("projection", 0),
                    cyl=ex.get("cyl"), **kw)


@pytest.mark.parametrize("name,seed", [("4x640x360cyl", 0), ("4x640x360cyl", 1), ("4x640x360cyl", 7),
                                       ("8x3840x2160cyl", 0)])
def test_cylindrical_geometry_matches_oracle(name, seed):
    rig, _ = rig_for_config(name, seed=seed)
    bands, rects = S.stitch_geometry(_cfg_of(rig))
    g = Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, projection=1, cyl=rig.extra["cyl"])
    assert [tuple(b) for b in bands.tolist()] == g.bands
    assert [tuple(map(tuple, r)) for r in rects.tolist()] == g.rects
    # bands lie inside both cameras' coverage and are not trivially small
    for p, (x0, x1, y0, y1) in enumerate(g.bands):
        assert x1 - x0 >= 16 and y1 - y0 >= rig.pano_h // 2
        for cam in (p, p + 1):
            xs = np.array([x0, x1 - 1, x0, x1 - 1], dtype=np.float64)
            ys = np.array([y0, y0, y1 - 1, y1 - 1], dtype=np.float64)
            sx, sy, sw = g.Hinv[cam].map(xs, ys)
            assert np.all(sw > 0) and np.all((sx >= 0) & (sx <= rig.cam_w[cam] - 1))


def test_cylindrical_config_checked():
    rig, _ = rig_for_config("4x640x360cyl", seed=0)
    with pytest.raises(S.StitchError) as ei:
        S.stitch_geometry(_cfg_of(rig) if False else S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h,
                                                               projection=1, cyl=(0.0, 0.0, 0.0)))
    assert "cyl_focal" in str(ei.value)
    with pytest.raises(S.StitchError) as ei:
        S.stitch_geometry(S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, projection=2,
                                   cyl=rig.extra["cyl"]))
    assert "projection" in str(ei.value)


def test_geometry_integer_translation():
    T = lambda tx, ty: np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])
    cfg = S.Config([200, 200], [100, 100], np.stack([T(0, 0), T(120, 0)]), 320, 100)
    bands, rects = S.stitch_geometry(cfg)
    assert bands.tolist() == [[120, 200, 0, 100]]
    assert rects.tolist() == [[[120, 200, 0, 100], [0, 80, 0, 100]]]


def _base_cfg(**over):
    rig, _ = rig_for_config("2x640x360", seed=0)
    kw = dict(cam_w=rig.cam_w, cam_h=rig.cam_h, H=rig.H, pano_w=rig.pano_w, pano_h=rig.pano_h)
    kw.update(over)
    return S.Config(**kw)


@pytest.mark.parametrize("over,needle", [
    (dict(window=0), "window"),
    (dict(window=17), "window"),
    (dict(lam=0.0), "lambda"),
    (dict(lam=0.5), "lambda"),
    (dict(max_flow=17.0), "max_flow"),
    (dict(max_flow=-1.0), "max_flow"),
    (dict(pano_pitch=1151), "pano_pitch"),
    (dict(pano_pitch=1136), "pano_pitch"),
    (dict(ref_cam=2), "ref_cam"),
    (dict(flags=64), "flag"),
    (dict(cam_pitch=[100, 1920]), "pitch"),
])
def test_invalid_config_rejected(over, needle):
    with pytest.raises(S.StitchError) as ei:
        S.stitch_geometry(_base_cfg(**over))
    assert ei.value.code == S.STITCH_EINVAL
    assert needle in str(ei.value)


def test_degenerate_rigs_rejected():
    T = lambda tx: np.array([[1.0, 0, tx], [0, 1.0, 0], [0, 0, 1.0]])
    # no overlap between the cameras
    with pytest.raises(S.StitchError, match="no overlap"):
        S.stitch_geometry(S.Config([100, 100], [50, 50], np.stack([T(0), T(150)]), 250, 50))
    # singular homography
    Hs = np.stack([T(0), np.zeros((3, 3))])
    with pytest.raises(S.StitchError, match="singular"):
        S.stitch_geometry(S.Config([100, 100], [50, 50], Hs, 200, 50))
    # non-finite entry
    Hn = np.stack([T(0), T(60)])
    Hn[1, 0, 2] = np.nan
    with pytest.raises(S.StitchError, match="non-finite"):
        S.stitch_geometry(S.Config([100, 100], [50, 50], Hn, 200, 50))
    # a single camera has no pair
    with pytest.raises(S.StitchError, match="n_cams"):
        S.stitch_geometry(S.Config([100], [50], T(0)[None], 100, 50))


def test_init_rejects_before_touching_the_device():
    with pytest.raises(S.StitchError) as ei:
        S.stitch_init(_base_cfg(window=99))
    assert ei.value.code == S.STITCH_EINVAL
    assert "window" in S.stitch_last_error(None)
