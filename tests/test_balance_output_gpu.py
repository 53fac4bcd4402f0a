"""GPU parity of the balance on the stitched image (STITCH_BALANCE_OUTPUT;
section 2.2 balances "the whole stitched image", Eq. 5-7): the knots of frame
T come from the pre-balance histogram of frame T - 1's panorama.

* Mosaic rig (two cameras at integer offsets over one image, zero flow,
  M = I): every fused value is an integer, so the library's histogram equals
  the histogram of the mosaic exactly, frame 0 comes out unbalanced and equal
  to the mosaic, and frame 1's knots are exactly the lambda quantiles of
  that histogram.
* A synthetic rig over a short sequence: histograms within a small fraction
  of the oracle's (the float32 and float64 fused values fall into different
  bins only near a bin's edge), knot means within a third of a level (one
  frame's knot one level apart), panoramas at the usual bar whenever the
  knots agree."""
import numpy as np
import pytest
import torch

from oracle import balance as bal
from oracle.pipeline import OracleStitcher
from paper_2308_09209_b300 import stitch as S

from gpu_common import FRAC_WITHIN_1, MAX_ABS, Pair, compare_pano, ensure_built

pytestmark = pytest.mark.gpu


def test_mosaic_histogram_exact_and_knots_from_it():
    ensure_built()
    rng = np.random.RandomState(4)
    h, w, off = 200, 400, 250
    mosaic = np.clip(rng.normal(120, 45, (h, off + w, 3)), 0, 255).astype(np.uint8)
    T = lambda tx: np.array([[1.0, 0, tx], [0, 1.0, 0], [0, 0, 1.0]])
    cfg = S.Config([w, w], [h, h], np.stack([T(0), T(off)]), off + w, h, max_flow=2.0,
                   flags=S.STITCH_BALANCE_OUTPUT)
    st = S.Stitcher(cfg)
    frames = [torch.from_numpy(mosaic[:, :w].copy()).cuda(), torch.from_numpy(mosaic[:, off:off + w].copy()).cuda()]
    x0, x1, y0, y1 = st.bands[0].tolist()
    fl = [torch.zeros((y1 - y0, x1 - x0, 2), dtype=torch.float32, device="cuda")]
    st.estimate_color(frames)
    pano = st.frame(frames, fl, fl)
    assert np.array_equal(pano.cpu().numpy()[:, :, :off + w].transpose(1, 2, 0), mosaic)   # frame 0 unbalanced
    hist = np.stack([np.bincount(mosaic[:, :, c].ravel(), minlength=256) for c in range(3)])
    assert np.array_equal(S.stitch_get_output_hist(st.ctx).astype(np.int64), hist)
    st.estimate_color(frames)
    m1, m2 = bal.knots(hist, 0.05)
    _, _, curve, _ = st.color()
    assert np.array_equal(curve["m1"], m1.astype(np.float32)) and np.array_equal(curve["m2"], m2.astype(np.float32))
    pano1 = st.frame(frames, fl, fl)
    o = OracleStitcher([T(0), T(off)], [w, w], [h, h], off + w, h, max_flow=2.0, flags=S.STITCH_BALANCE_OUTPUT)
    fr_np = [f.cpu().numpy() for f in frames]
    for _ in range(2):
        o.estimate_color(fr_np)
        planes, near, _ = o.frame(fr_np, [fl[0].cpu().numpy()], [fl[0].cpu().numpy()])
    r = compare_pano(pano1, planes, near, off + w)
    assert r["within1"] >= FRAC_WITHIN_1 and r["max"] <= MAX_ABS, r
    st.close()


def test_sequence_against_the_oracle():
    pr = Pair("2x640x360", seed=5, flags=S.STITCH_BALANCE_OUTPUT)
    for t in range(4):
        frames, fij, fji = pr.inputs(t)
        pr.st.estimate_color(frames)
        pano = pr.st.frame(frames, fij, fji)
        hist_g = S.stitch_get_output_hist(pr.st.ctx).astype(np.int64)
        fr_np = [f.cpu().numpy() for f in frames]
        pr.oracle.estimate_color(fr_np)
        _, _, curve, _ = pr.st.color()
        oc = pr.oracle.curve
        knots_agree = np.array_equal(curve["m1"], oc["m1"].astype(np.float32)) and \
            np.array_equal(curve["m2"], oc["m2"].astype(np.float32))
        assert np.all(np.abs(curve["m1"] - oc["m1"]) <= 1 / 3 + 1e-6) and \
            np.all(np.abs(curve["m2"] - oc["m2"]) <= 1 / 3 + 1e-6)
        planes, near, _ = pr.oracle.frame(fr_np, [f.cpu().numpy() for f in fij], [f.cpu().numpy() for f in fji])
        hist_o = pr.oracle.out_hist
        assert hist_g.sum() == hist_o.sum()
        assert np.abs(hist_g - hist_o).sum() <= 2e-3 * hist_o.sum(), np.abs(hist_g - hist_o).sum()
        if knots_agree:
            r = compare_pano(pano, planes, near, pr.rig.pano_w)
            assert r["within1"] >= FRAC_WITHIN_1 and r["max"] <= MAX_ABS, (t, r)
    pr.st.close()


def test_batch_rejects_balance_on_the_stitched_image():
    ensure_built()
    pr = Pair("2x640x360", seed=1, flags=S.STITCH_BALANCE_OUTPUT)
    with pytest.raises(S.StitchError) as ei:
        S.stitch_batch_create([pr.st.ctx])
    assert ei.value.code == S.STITCH_EINVAL
    pr.st.close()
