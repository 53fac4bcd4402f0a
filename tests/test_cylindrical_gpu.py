"""GPU parity of the cylindrical projection (the large-rig form): a small
cylindrical rig over a short sequence (full panorama), and the 8 x 3840 x 2160
cylindrical rig (window 7, flow up to 16 px, 12 moving objects) on sampled
pixels, both against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2308_09209_b300 import stitch as S

from gpu_common import FRAC_WITHIN_1, MAX_ABS, M_REL_TOL, Pair, compare_pano

pytestmark = pytest.mark.gpu


def _check_color(pr):
    _, Mg, _, _ = S.stitch_get_color(pr.st.ctx, pr.rig.n_cams)
    for k in range(pr.rig.n_cams):
        assert np.linalg.norm(Mg[k] - pr.oracle.M_cam[k]) <= M_REL_TOL * np.linalg.norm(pr.oracle.M_cam[k])


@pytest.mark.parametrize("flags", [0, S.STITCH_FP16_INTERMEDIATE])
def test_small_cylindrical_sequence_full_parity(flags):
    pr = Pair("4x640x360cyl", seed=2, flags=flags)
    for t in range(3):
        out = pr.step(t)
        r = compare_pano(out["pano"], out["planes"], out["near"], pr.rig.pano_w)
        assert r["within1"] >= FRAC_WITHIN_1 and r["max"] <= MAX_ABS, (t, r)
        _check_color(pr)
    pr.st.close()


def test_large_cylindrical_rig_sampled():
    pr = Pair("8x3840x2160cyl", seed=0, flags=S.STITCH_FP16_INTERMEDIATE)
    rng = np.random.default_rng(5)
    for t in range(2):
        out = pr.step(t, compare_pano=False)
    _check_color(pr)
    xs = rng.integers(0, pr.rig.pano_w, 60000)
    ys = rng.integers(0, pr.rig.pano_h, 60000)
    # half of the samples inside the blend bands, where the flow remap runs
    bands = pr.st.bands.tolist()
    for i in range(30000):
        x0, x1, y0, y1 = bands[i % len(bands)]
        xs[i] = rng.integers(x0, x1)
        ys[i] = rng.integers(y0, y1)
    vals, near = pr.oracle.pixels(out["fr_np"], [f.cpu().numpy() for f in out["fij"]],
                                  [f.cpu().numpy() for f in out["fji"]], xs, ys)
    g = out["pano"].cpu().numpy()[:, ys, xs].T.astype(np.int16)
    d = np.abs(g - vals.astype(np.int16)).max(1)[~near]
    assert (d <= 1).mean() >= FRAC_WITHIN_1 and d.max() <= MAX_ABS, (d.max(), (d <= 1).mean())
    pr.st.close()
