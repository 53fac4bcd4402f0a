"""GPU parity of the band optical flow (stitch_estimate_flow; section 3.2)
against the oracle (oracle/flow.py) on the same frames.

Bar: every cost is an integer, so a pixel's flow is identical on both sides
whenever the two luminance pyramids agree inside its matching windows. The
luminance differs only where the float32 pre-warp and the float64 one fall on
opposite sides of a rounding midpoint (up to about 2 pixels in 10^4 on the
cylinder, whose float32 ray arithmetic strays furthest), each such pixel
enters the 7 x 7 windows of 49 pixels, and the coarse levels spread a
changed choice to its children: at least 98 % of the band pixels must carry
bit-identical flows, and the others must stay within the search reach.

The two sources are also separated exactly: the library's luminance pyramid
(stitch_get_flow_luma) differs from the oracle's by one grey level at no more
than 0.1 % of the pixels, and the oracle's matcher run on the library's own
pyramid reproduces the library's flows bit for bit everywhere."""
import numpy as np
import pytest
import torch

from oracle.flow import pair_flows
from paper_2308_09209_b300 import stitch as S

from gpu_common import Pair, ensure_built

pytestmark = pytest.mark.gpu

FRAC_IDENTICAL = 0.98


def _gpu_flows(pr, frames):
    fij, fji = [], []
    for x0, x1, y0, y1 in pr.st.bands.tolist():
        fij.append(torch.full((y1 - y0, x1 - x0, 2), float("nan"), dtype=torch.float32, device="cuda"))
        fji.append(torch.full((y1 - y0, x1 - x0, 2), float("nan"), dtype=torch.float32, device="cuda"))
    S.stitch_estimate_flow(pr.st.ctx, frames, fij, fji)
    torch.cuda.synchronize()
    return [f.cpu().numpy() for f in fij], [f.cpu().numpy() for f in fji]


@pytest.mark.parametrize("config,seed", [("2x640x360", 0), ("4x640x360cyl", 1)])
def test_flow_matches_the_oracle(config, seed):
    pr = Pair(config, seed=seed)
    frames, _, _ = pr.inputs(2)
    gij, gji = _gpu_flows(pr, frames)
    oij, oji = pair_flows([f.cpu().numpy() for f in frames], pr.oracle.geom, pr.seq["max_flow"])
    reach = 4 * max(1, int(np.ceil(pr.seq["max_flow"] / 4))) + 2 + 1 + 0.5
    for g, o in zip(gij + gji, oij + oji):
        assert g.shape == o.shape and np.all(np.isfinite(g))
        same = np.all(g == o, axis=2)
        assert same.mean() >= FRAC_IDENTICAL, same.mean()
        assert np.all(np.abs(g) <= reach)
    pr.st.close()


def test_flow_feeds_the_stitch():
    """Estimated flows drive stitch_frame like supplied ones; the same call
    twice gives the same flows."""
    pr = Pair("2x640x360", seed=3)
    frames, _, _ = pr.inputs(0)
    a = _gpu_flows(pr, frames)
    b = _gpu_flows(pr, frames)
    assert all(np.array_equal(x, y) for x, y in zip(a[0] + a[1], b[0] + b[1]))
    fij = [torch.from_numpy(f).cuda() for f in a[0]]
    fji = [torch.from_numpy(f).cuda() for f in a[1]]
    pr.st.estimate_color(frames)
    pano = pr.st.frame(frames, fij, fji)
    torch.cuda.synchronize()
    assert pano.shape[0] == 3 and int(pano.max()) > 0
    pr.st.close()


def test_flow_argument_errors():
    ensure_built()
    pr = Pair("2x640x360", seed=0)
    frames, fij, fji = pr.inputs(0)
    with pytest.raises(S.StitchError) as ei:          # no flow estimated yet
        S.stitch_get_flow_luma(pr.st.ctx, 0, 0, 0)
    assert ei.value.code == S.STITCH_EINVAL
    S.stitch_estimate_flow(pr.st.ctx, frames, fij, fji)
    for pair, side, level in ((1, 0, 0), (0, 2, 0), (0, 0, 3), (-1, 0, 0)):
        with pytest.raises(S.StitchError):
            S.stitch_get_flow_luma(pr.st.ctx, pair, side, level)
    y2 = S.stitch_get_flow_luma(pr.st.ctx, 0, 1, 2)
    x0, x1, y0, y1 = pr.st.bands[0].tolist()
    assert y2.shape == ((y1 - y0 + 3) // 4, (x1 - x0 + 3) // 4)
    with pytest.raises(S.StitchError):
        S.stitch_estimate_flow(pr.st.ctx, frames, [0], fji)
    bad = torch.empty(fij[0].numel() * 4 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.StitchError):
        S.stitch_estimate_flow(pr.st.ctx, frames, [bad.data_ptr() + 4], fji)
    with pytest.raises(S.StitchError):
        S.stitch_estimate_flow(pr.st.ctx, frames[:1] + [0], fij, fji)
    pr.st.close()


@pytest.mark.parametrize("max_flow", [8.0, 4.0, 12.0, 16.0])
def test_flow_identical_where_both_prewarps_are_exact(max_flow):
    """Two cameras cropped from one rendered scene at integer offsets, the
    right one's content moved by (3, -2) against its homography: both
    pre-warps are exact copies of frame pixels, so both luminance pyramids,
    every integer cost and every float32 sub-pixel step agree, and the flows
    must be bit-identical everywhere. The search radius at the coarsest level
    is max_flow / 4: 1, 2, 3 and 4 (STITCH_MAX_FLOW) take one strip of three
    candidates per column, two overlapping strips, and three."""
    from oracle.pipeline import OracleStitcher
    from synth import Scene
    ensure_built()
    h, w, off, (dx, dy), m = 300, 640, 440, (3, -2), 8
    scene = Scene(off + w + 2 * m, h + 2 * m, n_objects=4, seed=11)
    ys, xs = torch.meshgrid(torch.arange(h + 2 * m, dtype=torch.float32), torch.arange(off + w + 2 * m,
                            dtype=torch.float32), indexing="ij")
    img = torch.round(scene.render(xs, ys, 0).clamp(0, 255)).to(torch.uint8)
    fa = img[m:m + h, m:m + w].contiguous()
    fb = img[m + dy:m + dy + h, m + off + dx:m + off + dx + w].contiguous()
    T = lambda tx: np.array([[1.0, 0, tx], [0, 1.0, 0], [0, 0, 1.0]])
    cfg = S.Config([w, w], [h, h], np.stack([T(0), T(off)]), off + w, h, max_flow=max_flow)
    st = S.Stitcher(cfg)
    frames = [fa.cuda(), fb.cuda()]
    x0, x1, y0, y1 = st.bands[0].tolist()
    gij = torch.full((y1 - y0, x1 - x0, 2), float("nan"), dtype=torch.float32, device="cuda")
    gji = torch.full_like(gij, float("nan"))
    S.stitch_estimate_flow(st.ctx, frames, [gij], [gji])
    torch.cuda.synchronize()
    o = OracleStitcher(cfg.H, cfg.cam_w, cfg.cam_h, cfg.pano_w, cfg.pano_h, max_flow=max_flow)
    oij, oji = pair_flows([fa.numpy(), fb.numpy()], o.geom, max_flow)
    g1, g2 = gij.cpu().numpy(), gji.cpu().numpy()
    assert np.array_equal(g1, oij[0]) and np.array_equal(g2, oji[0])
    if max_flow != 8.0:
        st.close()
        return
    # away from the band's border the match is the known shift within the
    # sub-pixel step (the parabola through asymmetric costs moves it off the
    # integer by up to half a pixel), in one direction or the other: the
    # median over the core is the shift, and most vectors sit within half a
    # pixel of it (block matching cannot see the shift on the scene's flat
    # areas; the GPU and the oracle agree bit for bit, so the share is fixed
    # for this seeded scene: 0.71)
    core = (slice(m, -m), slice(m, -m))
    s = np.array([dx, dy], np.float32)
    near = lambda f, v: np.all(np.abs(f[core] - v) <= 0.5, axis=-1)
    for g in (g1, g2):
        med = np.median(g[core].reshape(-1, 2), axis=0)
        assert np.all(np.abs(med - s) <= 0.5) or np.all(np.abs(med + s) <= 0.5), med
        assert max(np.mean(near(g, s)), np.mean(near(g, -s))) > 0.6
    st.close()


def test_flow_matches_the_oracle_at_full_size():
    """The benchmark's rig (bands about 400 x 1066): band 0, both directions,
    with the same bar as the small rigs."""
    from oracle.flow import band_prewarp, flow
    pr = Pair("4x1920x1080", seed=0)
    frames, _, _ = pr.inputs(2)
    gij, gji = _gpu_flows(pr, frames)
    fr = [f.cpu().numpy() for f in frames]
    band = pr.oracle.geom.bands[0]
    Pi = band_prewarp(fr[0], pr.oracle.geom, 0, band)
    Pj = band_prewarp(fr[1], pr.oracle.geom, 1, band)
    oij, oji = flow(Pi, Pj, pr.seq["max_flow"]), flow(Pj, Pi, pr.seq["max_flow"])
    reach = 4 * max(1, int(np.ceil(pr.seq["max_flow"] / 4))) + 2 + 1 + 0.5
    for g, o in ((gij[0], oij), (gji[0], oji)):
        assert g.shape == o.shape and np.all(np.isfinite(g))
        same = np.all(g == o, axis=2)
        assert same.mean() >= FRAC_IDENTICAL, same.mean()
        assert np.all(np.abs(g) <= reach)
    pr.st.close()


@pytest.mark.parametrize("config,seed,t", [("4x1920x1080", 0, 2), ("4x640x360cyl", 1, 0)])
def test_matcher_exact_on_the_librarys_luminance(config, seed, t):
    """The two sources of difference, separated. (1) Luminance: the library's
    float32 pre-warp rounds to the oracle's integer luminance except at a few
    pixels, by one grey level at most, and its pyramid levels 1 and 2 are the
    exact integer reductions of its own level 0. (2) Matching: every cost is an
    integer and the sub-pixel step is float32 on both sides, so the oracle's
    matcher (section 3.2 steps 3-5) run on the library's own pyramids must give
    the library's flows bit for bit, everywhere, in both directions (band 0;
    the benchmark rig at full size and the small cylindrical rig)."""
    from oracle.flow import band_prewarp, downsample, flow_from_pyramids, luminance
    pr = Pair(config, seed=seed)
    frames, _, _ = pr.inputs(t)
    gij, gji = _gpu_flows(pr, frames)
    fr = [f.cpu().numpy() for f in frames]
    geom = pr.oracle.geom
    band = geom.bands[0]
    pyr = {}
    for side in (0, 1):
        levels = [S.stitch_get_flow_luma(pr.st.ctx, 0, side, lev).astype(np.int64) for lev in range(3)]
        Yo = luminance(band_prewarp(fr[side], geom, side, band))
        d = np.abs(levels[0] - Yo)
        assert levels[0].shape == Yo.shape and d.max() <= 1 and (d > 0).mean() <= 1e-3, (d.max(), (d > 0).mean())
        assert np.array_equal(levels[1], downsample(levels[0]))
        assert np.array_equal(levels[2], downsample(levels[1]))
        pyr[side] = levels
    mf = pr.seq["max_flow"]
    assert np.array_equal(gij[0], flow_from_pyramids(pyr[0], pyr[1], mf))
    assert np.array_equal(gji[0], flow_from_pyramids(pyr[1], pyr[0], mf))
    pr.st.close()
