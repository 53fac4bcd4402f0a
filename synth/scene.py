"""Procedural scene and per-camera frame rendering.

The scene lives on the panorama plane and is evaluated analytically at any
continuous point: 64 Gaussian colour blobs, 4 octaves of value noise (random
lattice values, smoothstep interpolation) and optional moving rectangles with
striped textures that translate with constant velocity. A camera frame is the
scene sampled at G_k (u, v, 1) for every camera pixel, then pushed through
that camera's colour cast, per-channel gain, gamma and offset and rounded to
uint8 (packed RGB, HWC).
"""
from __future__ import annotations

import math

import numpy as np
import torch


class Scene:
    def __init__(self, extent_w, extent_h, n_blobs=64, octaves=4, n_objects=0,
                 seed=0, object_speed=6.0):
        rng = np.random.RandomState(seed + 7919)
        self.W = float(extent_w)
        self.Hh = float(extent_h)
        margin = 0.1 * max(extent_w, extent_h)
        self.blob_c = np.stack([rng.uniform(-margin, extent_w + margin, n_blobs),
                                rng.uniform(-margin, extent_h + margin, n_blobs)], 1)
        self.blob_s = rng.uniform(0.03, 0.25, n_blobs) * extent_h
        self.blob_rgb = rng.uniform(-55.0, 85.0, (n_blobs, 3))
        self.base = rng.uniform(70.0, 110.0, 3)
        self.oct = []
        cell = max(extent_h / 3.0, 16.0)
        for o in range(octaves):
            gw = int(math.ceil((extent_w + 2 * margin) / cell)) + 3
            gh = int(math.ceil((extent_h + 2 * margin) / cell)) + 3
            lat = rng.uniform(-1.0, 1.0, (gh, gw, 3))
            self.oct.append((cell, margin, lat, 38.0 * 0.55 ** o))
            cell /= 2.0
        self.objs = []
        for _ in range(n_objects):
            w = rng.uniform(0.04, 0.12) * extent_h * 2
            h = rng.uniform(0.04, 0.12) * extent_h * 2
            p0 = (rng.uniform(0, extent_w), rng.uniform(0.2, 0.8) * extent_h)
            v = (rng.uniform(-object_speed, object_speed), rng.uniform(-object_speed / 3, object_speed / 3))
            c1 = rng.uniform(0, 255, 3)
            c2 = rng.uniform(0, 255, 3)
            period = rng.uniform(6.0, 24.0)
            ang = rng.uniform(0, math.pi)
            self.objs.append((w, h, p0, v, c1, c2, period, ang))

    def render(self, X: torch.Tensor, Y: torch.Tensor, t: int = 0) -> torch.Tensor:
        """Scene colour (float32, [..., 3], roughly 0..255) at world points (X, Y)."""
        dev = X.device
        out = torch.empty(X.shape + (3,), dtype=torch.float32, device=dev)
        out[...] = torch.tensor(self.base, dtype=torch.float32, device=dev)
        for (cx, cy), s, rgb in zip(self.blob_c, self.blob_s, self.blob_rgb):
            g = torch.exp(-((X - float(cx)) ** 2 + (Y - float(cy)) ** 2) * (0.5 / float(s) ** 2))
            out += g[..., None] * torch.tensor(rgb, dtype=torch.float32, device=dev)
        for cell, margin, lat, amp in self.oct:
            L = torch.tensor(lat, dtype=torch.float32, device=dev)
            gx = (X + margin) / cell
            gy = (Y + margin) / cell
            ix = torch.floor(gx)
            iy = torch.floor(gy)
            fx = gx - ix
            fy = gy - iy
            fx = fx * fx * (3 - 2 * fx)
            fy = fy * fy * (3 - 2 * fy)
            ix = ix.long().clamp(0, L.shape[1] - 2)
            iy = iy.long().clamp(0, L.shape[0] - 2)
            v00 = L[iy, ix]
            v10 = L[iy, ix + 1]
            v01 = L[iy + 1, ix]
            v11 = L[iy + 1, ix + 1]
            top = v00 + (v10 - v00) * fx[..., None]
            bot = v01 + (v11 - v01) * fx[..., None]
            out += amp * (top + (bot - top) * fy[..., None])
        for (w, h, p0, v, c1, c2, period, ang) in self.objs:
            cx = (p0[0] + v[0] * t) % self.W
            cy = p0[1] + v[1] * t
            cy = cy % self.Hh
            inside = ((X - cx).abs() < w / 2) & ((Y - cy).abs() < h / 2)
            if not bool(inside.any()):
                continue
            phase = ((X - cx) * math.cos(ang) + (Y - cy) * math.sin(ang)) / period
            stripe = (torch.floor(phase).long() % 2 == 0)
            col = torch.where(stripe[..., None],
                              torch.tensor(c1, dtype=torch.float32, device=dev),
                              torch.tensor(c2, dtype=torch.float32, device=dev))
            out = torch.where(inside[..., None], col, out)
        return out


def _photometric(rgb: torch.Tensor, gain, gamma, offset, cast) -> torch.Tensor:
    dev = rgb.device
    c = rgb.clamp(0.0, 255.0)
    if not np.allclose(cast, np.eye(3)):
        c = (c @ torch.tensor(cast.T, dtype=torch.float32, device=dev)).clamp(0.0, 255.0)
    g = torch.tensor(gain, dtype=torch.float32, device=dev)
    gm = torch.tensor(gamma, dtype=torch.float32, device=dev)
    of = torch.tensor(offset, dtype=torch.float32, device=dev)
    c = 255.0 * g * torch.pow(c / 255.0, gm) + of
    return torch.round(c.clamp(0.0, 255.0)).to(torch.uint8)


def render_camera_frames(rig, scene: Scene, t: int = 0, device="cpu",
                         photometric=True, rows_per_chunk=540, noise=0.0, noise_seed=0):
    """Render every camera's frame at time t: a list of uint8 [h, w, 3] tensors.
    noise > 0 adds seeded Gaussian sensor noise of that standard deviation
    (grey levels) to the scene radiance of every pixel, drawn independently
    per frame, camera and row chunk (seeded from noise_seed, t, k)."""
    frames = []
    for k in range(rig.n_cams):
        w, h = rig.cam_w[k], rig.cam_h[k]
        G = rig.G[k]
        img = torch.empty((h, w, 3), dtype=torch.uint8, device=device)
        u = torch.arange(w, dtype=torch.float64, device=device)
        for r0 in range(0, h, rows_per_chunk):
            r1 = min(h, r0 + rows_per_chunk)
            v = torch.arange(r0, r1, dtype=torch.float64, device=device)
            V, U = torch.meshgrid(v, u, indexing="ij")
            if rig.extra.get("projection", 0) == 1:
                # cylindrical rig: the ray of each pixel, unrolled on the cylinder
                f, cx, cy = rig.extra["cyl"]
                d0 = G[0, 0] * U + G[0, 1] * V + G[0, 2]
                d1 = G[1, 0] * U + G[1, 1] * V + G[1, 2]
                d2 = G[2, 0] * U + G[2, 1] * V + G[2, 2]
                X = (cx + f * torch.atan2(d0, d2)).float()
                Y = (cy + f * d1 / torch.sqrt(d0 * d0 + d2 * d2)).float()
            else:
                den = G[2, 0] * U + G[2, 1] * V + G[2, 2]
                X = ((G[0, 0] * U + G[0, 1] * V + G[0, 2]) / den).float()
                Y = ((G[1, 0] * U + G[1, 1] * V + G[1, 2]) / den).float()
            rgb = scene.render(X, Y, t)
            if noise > 0:
                gen = torch.Generator(device=device)
                gen.manual_seed(((int(noise_seed) * 1000003 + int(t)) * 64 + k) * 4096 + r0 // rows_per_chunk)
                rgb = rgb + float(noise) * torch.randn(rgb.shape, generator=gen, device=device, dtype=rgb.dtype)
            if photometric:
                img[r0:r1] = _photometric(rgb, rig.gain[k], rig.gamma[k], rig.offset[k], rig.cast[k])
            else:
                img[r0:r1] = torch.round(rgb.clamp(0, 255)).to(torch.uint8)
        frames.append(img)
    return frames
