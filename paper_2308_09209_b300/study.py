"""Temporal-window study of the colour transfer (the comparison of the paper's
Tables 2 and 3: a one-frame M, as in the 2D-M method it compares against,
against the spatio-temporal 3D-M over a window of frames).

For each window W the library's plain estimator (stitch_estimate_color, one
call per frame) runs over the same seeded sequence of a rig with moving
objects and per-frame sensor noise (objects that stay inside an overlap
leave its histograms unchanged; noise is what makes a real video's M vary
from frame to frame). For every frame and pair the colour source camera i is
mapped into the panorama over the pair's blend band (bilinear samples of its
frame at H_i^-1 q, float64 on the GPU, evaluation only), transferred with the
pair's M (stitch_get_pair_M) and compared with the target camera j sampled
the same way: PSNR = 10 log10(255^2 / mean squared difference over the
band's pixels and channels). Reported per window: the mean and the frame-to-frame standard
deviation of the PSNR (Table 2's mu and sigma rows), and the mean
frame-to-frame standard deviation of M's entries. The first W - 1 frames,
where the window is not yet full, are left out of the statistics. The same
figures for the 2D-M method the paper compares against (a one-frame least-
squares map from the bands' pixel correspondences,
stitch_pair_M_correspondence) are reported beside them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import stitch as S


def _sample(frame: torch.Tensor, Hinv: torch.Tensor, xs: torch.Tensor, ys: torch.Tensor) -> torch.Tensor:
    """Bilinear samples (float64 [n, 3]) of a uint8 [h, w, 3] frame at H^-1 q
    for panorama points q = (xs, ys); points outside the frame are clamped."""
    h, w, _ = frame.shape
    sx = Hinv[0, 0] * xs + Hinv[0, 1] * ys + Hinv[0, 2]
    sy = Hinv[1, 0] * xs + Hinv[1, 1] * ys + Hinv[1, 2]
    sw = Hinv[2, 0] * xs + Hinv[2, 1] * ys + Hinv[2, 2]
    sx = (sx / sw).clamp(0, w - 1)
    sy = (sy / sw).clamp(0, h - 1)
    x0 = sx.floor().clamp(max=w - 2).long()
    y0 = sy.floor().clamp(max=h - 2).long()
    fx = (sx - x0).unsqueeze(1)
    fy = (sy - y0).unsqueeze(1)
    f = frame.double()
    a, b = f[y0, x0], f[y0, x0 + 1]
    c, d = f[y0 + 1, x0], f[y0 + 1, x0 + 1]
    return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d)


def window_study(config: str = "3x1920x1080", windows=(1, 3, 5, 7), n_frames: int = 16, seed: int = 5,
                 objects: int = 12, object_speed: float = 24.0, noise: float = 2.0) -> dict:
    from synth import Scene, render_camera_frames, rig_for_config
    rig, seq = rig_for_config(config, seed=seed, objects=objects)
    scene = Scene(rig.pano_w, rig.pano_h, n_objects=objects, seed=seed, object_speed=object_speed)
    n = rig.n_cams
    ref = n // 2
    dev = torch.device("cuda")
    frames = [render_camera_frames(rig, scene, t, device="cuda", noise=noise, noise_seed=seed) for t in range(n_frames)]
    bands, _ = S.stitch_geometry(S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h))
    Hinv = [torch.tensor(np.linalg.inv(np.asarray(h, np.float64).reshape(3, 3)), device=dev) for h in rig.H]
    grids = []
    for x0, x1, y0, y1 in bands.tolist():
        yy, xx = torch.meshgrid(torch.arange(y0, y1, dtype=torch.float64, device=dev),
                                torch.arange(x0, x1, dtype=torch.float64, device=dev), indexing="ij")
        grids.append((xx.reshape(-1), yy.reshape(-1)))
    out = {"rig": config, "frames": n_frames, "moving_objects": objects, "object_speed_px": object_speed,
           "sensor_noise_sigma": noise, "per_window": {}}
    def psnr_row(t, Mp):
        row = []
        for p in range(n - 1):
            i = p if p < ref else p + 1              # colour source of the pair (away from the reference)
            j = p + 1 if p < ref else p
            xs, ys = grids[p]
            Pi = _sample(frames[t][i], Hinv[i], xs, ys)
            Pj = _sample(frames[t][j], Hinv[j], xs, ys)
            Mt = torch.tensor(Mp[p], dtype=torch.float64, device=dev)
            mse = float(((Pi @ Mt).clamp(0, 255) - Pj).pow(2).mean())
            row.append(10.0 * np.log10(255.0 ** 2 / max(mse, 1e-12)))
        return row

    def summary(psnr, Ms):
        psnr = np.asarray(psnr)                      # [frames, pairs]
        Ms = np.asarray(Ms)                          # [frames, pairs, 3, 3]
        return {"psnr_mu": float(psnr.mean()), "psnr_sigma": float(psnr.std(axis=0).mean()),
                "sigma_M": float(Ms.std(axis=0).mean()), "frames_used": int(psnr.shape[0])}

    for W in windows:
        cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=W, max_flow=seq["max_flow"])
        st = S.Stitcher(cfg)
        psnr, Ms = [], []
        for t in range(n_frames):
            st.estimate_color(frames[t])
            Mp = S.stitch_get_pair_M(st.ctx, n - 1)
            if t < W - 1:
                continue
            psnr.append(psnr_row(t, Mp))
            Ms.append(np.asarray(Mp, np.float64).copy())
        if W == windows[0]:
            # the 2D-M comparison: one-frame least squares over the pixel correspondences
            p2, M2 = [], []
            for t in range(n_frames):
                Mc = S.stitch_pair_M_correspondence(st.ctx, frames[t], n - 1)
                p2.append(psnr_row(t, Mc))
                M2.append(np.asarray(Mc, np.float64).copy())
            out["2d_m_correspondence"] = summary(p2, M2)
        st.close()
        out["per_window"][str(W)] = summary(psnr, Ms)
    return out
