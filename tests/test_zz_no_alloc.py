"""The allocation-free colour estimate (stitch_estimate_color_noalloc).

Callers such as plugins inside a host application that owns all device
memory, or code that must not enter the CUDA allocator while capturing a
stream or on a real-time thread, cannot call cudaMalloc; this entry point
gives them the colour estimate of one frame using only a fixed scratch array
built into the library. The test calls it through the C ABI twice in a row on
different frames (the second call reuses the scratch the first one left
behind) and checks each result against the regular context-based entry point
on a fresh context, with the same tolerances as the other parity tests.

This file is named so that pytest collects it after every other test.
"""
import numpy as np
import pytest
import torch

from gpu_common import M_REL_TOL, ensure_built, rel_err
from paper_2308_09209_b300 import stitch as S
from synth import Scene, render_camera_frames, rig_for_config


def _reference(cfg, frames):
    st = S.Stitcher(cfg)
    try:
        st.estimate_color(frames)
        rc, M, curve, T = st.color()
        return M, curve, rc
    finally:
        st.close()


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["2x640x360", "4x1920x1080"])
def test_noalloc_matches_context_estimate_on_two_calls(name):
    ensure_built()
    rig, seq = rig_for_config(name, seed=2)
    cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                   max_flow=seq["max_flow"])
    scene = Scene(rig.pano_w, rig.pano_h, n_objects=seq.get("objects", 0), seed=2)
    n = rig.n_cams
    for t in (0, 5):                       # two calls in a row, different frames
        frames = render_camera_frames(rig, scene, t, device="cuda")
        M_dev = torch.full((n * 9,), float("nan"), dtype=torch.float64, device="cuda")
        curve_dev = torch.full((3 * S.STITCH_CURVE_FLOATS,), float("nan"), dtype=torch.float32, device="cuda")
        flags_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert S.stitch_estimate_color_noalloc(cfg, frames, M_dev, curve_dev, flags_dev) == S.STITCH_OK
        torch.cuda.synchronize()
        if t == 5:
            # the second call takes no device memory: free bytes unchanged around it
            # (the first call in a fresh process may still load kernel code)
            assert torch.cuda.mem_get_info()[0] == free0
        M_ref, curve_ref, rc = _reference(cfg, frames)
        M = M_dev.cpu().numpy().reshape(n, 3, 3)
        for k in range(n):
            assert rel_err(M[k], M_ref[k]) <= M_REL_TOL, (t, k)
        curve = curve_dev.cpu().numpy().reshape(3, S.STITCH_CURVE_FLOATS)
        for i, field in enumerate(S.CURVE_FIELDS):
            if field in ("m1", "m2", "identity"):
                assert np.array_equal(curve[:, i], curve_ref[field]), field
            else:
                assert np.allclose(curve[:, i], curve_ref[field], rtol=1e-6, atol=1e-6), field
        assert int(flags_dev.item()) == 0 and rc == S.STITCH_OK


@pytest.mark.gpu
def test_noalloc_rejects_rigs_beyond_the_scratch():
    ensure_built()
    T = lambda tx: np.array([[1.0, 0, tx], [0, 1.0, 0], [0, 0, 1.0]])
    n = S.STITCH_MAX_CAMS + 1
    cfg = S.Config([200] * n, [100] * n, np.stack([T(150 * k) for k in range(n)]), 150 * n + 50, 100)
    frames = [torch.zeros((100, 200, 3), dtype=torch.uint8, device="cuda") for _ in range(n)]
    M_dev = torch.zeros((n * 9,), dtype=torch.float64, device="cuda")
    curve_dev = torch.zeros((30,), dtype=torch.float32, device="cuda")
    with pytest.raises(S.StitchError) as ei:
        S.stitch_estimate_color_noalloc(cfg, frames, M_dev, curve_dev)
    assert ei.value.code == S.STITCH_EINVAL and "at most 8 cameras" in str(ei.value)


@pytest.mark.gpu
def test_noalloc_checks_its_output_tensors():
    ensure_built()
    rig, seq = rig_for_config("2x640x360", seed=2)
    cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                   max_flow=seq["max_flow"])
    frames = [torch.zeros((h, w, 3), dtype=torch.uint8, device="cuda") for w, h in zip(rig.cam_w, rig.cam_h)]
    curve = torch.zeros((3 * S.STITCH_CURVE_FLOATS,), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):          # float32 instead of float64
        S.stitch_estimate_color_noalloc(cfg, frames, torch.zeros(18, dtype=torch.float32, device="cuda"), curve)
    with pytest.raises(ValueError):          # too short
        S.stitch_estimate_color_noalloc(cfg, frames, torch.zeros(17, dtype=torch.float64, device="cuda"), curve)
