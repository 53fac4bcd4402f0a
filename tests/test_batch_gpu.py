"""GPU tests of the fuse tile shapes, the autotuner and the batched launch of
several rigs: every shape and the batch must give exactly what one rig
stitched alone gives, and the batch's outputs are checked against the FP64
oracle on sampled pixels."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from oracle.pipeline import OracleStitcher
from paper_2308_09209_b300 import stitch as S
from synth import BATCH_RIGS, Scene, render_camera_frames, rig_for_config

from gpu_common import (FRAC_WITHIN_1, MAX_ABS, M_REL_TOL, Pair, compare_pano, ensure_built, flows_for,
                        oracle_frame_parallel)

pytestmark = pytest.mark.gpu


def test_every_tile_shape_gives_the_same_panorama():
    ensure_built()
    pr = Pair("4x1920x1080", seed=1)
    frames, fij, fji = pr.inputs(0)
    pr.st.estimate_color(frames)
    ref = pr.st.frame(frames, fij, fji).clone()
    fits = 0
    for shape in range(S.STITCH_TILE_SHAPES):
        try:
            S.stitch_set_tile_shape(pr.st.ctx, shape)
        except S.StitchError:
            continue
        fits += 1
        assert S.stitch_tile_shape(pr.st.ctx)[1] == S.TILE_SHAPES[shape]
        out = pr.st.frame(frames, fij, fji)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"shape {S.TILE_SHAPES[shape]}"
    assert fits >= 3
    shape, ms = S.stitch_autotune(pr.st.ctx, frames, fij, fji, pr.st.new_pano(), reps=3)
    # the fastest shape, or the default one when none beats it by more than 5 %
    fastest = ms[ms > 0].min()
    assert ms[shape] > 0 and (ms[shape] == fastest or (shape == 0 and fastest > 0.95 * ms[0])), ms
    assert S.stitch_tile_shape(pr.st.ctx)[0] == shape
    out = pr.st.frame(frames, fij, fji)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    pr.st.close()


def _rig_inputs(names, seeds, n_frames):
    rigs = []
    for name, seed in zip(names, seeds):
        rig, seq = rig_for_config(name, seed=seed)
        scene = Scene(rig.pano_w, rig.pano_h, n_objects=seq.get("objects", 0), seed=seed)
        cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                       max_flow=seq["max_flow"])
        st = S.Stitcher(cfg)
        frames = [render_camera_frames(rig, scene, t, device="cuda") for t in range(n_frames)]
        flows = [flows_for(st.bands, seq["max_flow"], seed, t) for t in range(n_frames)]
        rigs.append(dict(rig=rig, seq=seq, cfg=cfg, st=st, frames=frames, flows=flows, seed=seed))
    return rigs


def _flat(rigs, n_frames):
    fr, fij, fji, pano = [], [], [], []
    for t in range(n_frames):
        for r in rigs:
            fr += r["frames"][t]
            fij += r["flows"][t][0]
            fji += r["flows"][t][1]
            pano.append(r["panos"][t])
    return fr, fij, fji, pano


def _alone(r, n_frames):
    """The same frames through a fresh single-rig context (stitch_sequence)."""
    st = S.Stitcher(r["cfg"])
    outs = [st.new_pano() for _ in range(n_frames)]
    S.stitch_sequence(st.ctx, n_frames, [f for t in range(n_frames) for f in r["frames"][t]],
                      [f for t in range(n_frames) for f in r["flows"][t][0]],
                      [f for t in range(n_frames) for f in r["flows"][t][1]], outs)
    torch.cuda.synchronize()
    st.close()
    return outs


@pytest.mark.parametrize("fp16", [False, True])
def test_batch_equals_each_rig_alone(fp16):
    ensure_built()
    n_frames = 5
    rigs = _rig_inputs(["2x640x360", "3x1920x1080", "2x1280x720"], [0, 1, 2], n_frames)
    if fp16:
        for r in rigs:
            r["st"].close()
            r["cfg"].flags = S.STITCH_FP16_INTERMEDIATE
            r["st"] = S.Stitcher(r["cfg"])
    # a different tile shape per rig: the persistent kernels run every rig's
    # tiles with that rig's shape
    want = []
    for r, sh in zip(rigs, (2, 1, 3)):
        try:
            S.stitch_set_tile_shape(r["st"].ctx, sh)
        except S.StitchError:
            pass
        want.append(S.stitch_tile_shape(r["st"].ctx)[0])
    assert len(set(want)) >= 2
    for r in rigs:
        r["panos"] = [r["st"].new_pano() for _ in range(n_frames)]
    b = S.stitch_batch_create([r["st"].ctx for r in rigs])
    assert S.stitch_batch_tile_shapes(b) == want
    fr, fij, fji, pano = _flat(rigs, n_frames)
    S.stitch_batch_sequence(b, n_frames, fr, fij, fji, pano)
    torch.cuda.synchronize()
    for r in rigs:
        alone = _alone(r, n_frames)
        for t in range(n_frames):
            assert torch.equal(r["panos"][t], alone[t]), (r["cfg"].cam_w, t)
    # a second call replays the recorded graph and continues the colour state
    for r in rigs:
        r["panos"] = [r["st"].new_pano() for _ in range(n_frames)]
    fr, fij, fji, pano = _flat(rigs, n_frames)
    S.stitch_batch_sequence(b, n_frames, fr, fij, fji, pano)
    torch.cuda.synchronize()
    for r in rigs:
        assert S.stitch_get_color(r["st"].ctx, len(r["rig"].cam_w))[3] == 2 * n_frames
    S.stitch_batch_destroy(b)
    for r in rigs:
        r["st"].close()


def test_full_batch_against_the_oracle_every_pixel():
    """The four rigs of the batched workload (a mixed 6x1080p + 2x720p rig,
    3x1080p, 4x2160p, 2x720p), FP16 intermediates, tile shape autotuned: every
    pixel of every rig's panorama against the FP64 oracle's whole panorama,
    and its pair matrices against the oracle's."""
    ensure_built()
    n_frames = 2
    rigs = _rig_inputs(BATCH_RIGS, [10, 11, 12, 13], n_frames)
    for r in rigs:
        r["st"].close()
        r["cfg"].flags = S.STITCH_FP16_INTERMEDIATE
        r["st"] = S.Stitcher(r["cfg"])
        r["panos"] = [r["st"].new_pano() for _ in range(n_frames)]
    b = S.stitch_batch_create([r["st"].ctx for r in rigs])
    fr, fij, fji, pano = _flat(rigs, 1)
    shapes, ms = S.stitch_batch_autotune(b, fr, fij, fji, pano, reps=2)
    assert S.stitch_batch_tile_shapes(b) == shapes and ms.shape == (len(rigs), S.STITCH_TILE_SHAPES)
    for r, sh in enumerate(shapes):
        # every rig's chosen shape is its fastest fitting one (the other rigs at their shapes then),
        # or the default one when none beats it by more than 5 %
        fastest = ms[r][ms[r] > 0].min()
        assert ms[r, sh] > 0 and (ms[r, sh] == fastest or (sh == 0 and fastest > 0.95 * ms[r, 0])), ms[r]
    fr, fij, fji, pano = _flat(rigs, n_frames)
    S.stitch_batch_sequence(b, n_frames, fr, fij, fji, pano)
    torch.cuda.synchronize()
    for r in rigs:
        rig, seq = r["rig"], r["seq"]
        o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                           max_flow=seq["max_flow"], flags=S.STITCH_FP16_INTERMEDIATE)
        for t in range(n_frames):
            fr_np = [f.cpu().numpy() for f in r["frames"][t]]
            o.estimate_color(fr_np)
        t = n_frames - 1
        view = SimpleNamespace(rig=rig, oracle=o, proj=dict(projection=0, cyl=None))
        planes, near = oracle_frame_parallel(view, [f.cpu().numpy() for f in r["frames"][t]],
                                             [f.cpu().numpy() for f in r["flows"][t][0]],
                                             [f.cpu().numpy() for f in r["flows"][t][1]])
        rep = compare_pano(r["panos"][t], planes, near, rig.pano_w)
        assert rep["within1"] >= FRAC_WITHIN_1 and rep["max"] <= MAX_ABS, (rig.cam_w, rep)
        assert rep["n"] + rep["n_near"] == rig.pano_w * rig.pano_h
        Mp = S.stitch_get_pair_M(r["st"].ctx, len(rig.cam_w) - 1)
        for p in range(len(rig.cam_w) - 1):
            assert np.linalg.norm(Mp[p] - o.M_pair[p]) <= M_REL_TOL * np.linalg.norm(o.M_pair[p])
    S.stitch_batch_destroy(b)
    for r in rigs:
        r["st"].close()


def test_batch_argument_errors():
    ensure_built()
    rigs = _rig_inputs(["2x640x360", "2x640x360"], [0, 1], 1)
    with pytest.raises(S.StitchError):
        S.stitch_batch_create([rigs[0]["st"].ctx, rigs[0]["st"].ctx])
    rigs[1]["st"].close()
    cfg = rigs[1]["cfg"]
    cfg.flags = S.STITCH_FP16_INTERMEDIATE
    rigs[1]["st"] = S.Stitcher(cfg)
    with pytest.raises(S.StitchError):
        S.stitch_batch_create([rigs[0]["st"].ctx, rigs[1]["st"].ctx])
    for r in rigs:
        r["st"].close()
