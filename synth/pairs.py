"""Seeded training pairs for the learned colour estimator.

A pair is two patches of the same procedural scene content (a random crop,
side j shifted by up to ``max_shift`` pixels) seen through two independent
photometric responses, each drawn as in the rig generator: per channel gain
U(0.8, 1.2), gamma U(0.9, 1.1), offset U(-8, 8), and a colour cast with
off-diagonal entries U(-cast, cast) (rows renormalised to sum to 1). Side i is
the camera to correct, side j the reference. Output: uint8 tensor
[n, 2, patch_h, patch_w, 3] (packed RGB per patch) on ``device``.

This module only draws inputs; it holds none of the estimator's arithmetic.
"""
from __future__ import annotations

import numpy as np
import torch

from .scene import Scene


def _responses(rng, n, cast):
    gain = rng.uniform(0.8, 1.2, (n, 3))
    gamma = rng.uniform(0.9, 1.1, (n, 3))
    offset = rng.uniform(-8.0, 8.0, (n, 3))
    C = np.tile(np.eye(3), (n, 1, 1))
    if cast > 0:
        off = rng.uniform(-cast, cast, (n, 3, 3))
        off[:, [0, 1, 2], [0, 1, 2]] = 0.0
        C = C + off
        C = C / C.sum(axis=2, keepdims=True)
    return gain, gamma, offset, C


def apply_response(rgb: torch.Tensor, gain, gamma, offset, C) -> torch.Tensor:
    """rgb: float [n, ..., 3] scene colours; per-item response parameters
    (numpy [n, 3] / [n, 3, 3]). Returns uint8 of the same shape."""
    dev = rgb.device
    n = rgb.shape[0]
    shp = (n,) + (1,) * (rgb.dim() - 2) + (3,)
    c = rgb.clamp(0.0, 255.0)
    Ct = torch.tensor(np.transpose(C, (0, 2, 1)), dtype=torch.float32, device=dev)   # v' = v C^T
    c = torch.einsum("n...c,ncd->n...d", c, Ct).clamp(0.0, 255.0)
    g = torch.tensor(gain, dtype=torch.float32, device=dev).view(shp)
    gm = torch.tensor(gamma, dtype=torch.float32, device=dev).view(shp)
    of = torch.tensor(offset, dtype=torch.float32, device=dev).view(shp)
    c = 255.0 * g * torch.pow(c / 255.0, gm) + of
    return torch.round(c.clamp(0.0, 255.0)).to(torch.uint8)


def make_pairs(n, patch_w=96, patch_h=64, seed=0, device="cpu", n_scenes=16, scene_w=1152, scene_h=360,
               max_shift=3, cast=0.05, chunk=4096):
    """n seeded pairs (see the module docstring) and their response
    parameters: (pairs uint8 [n, 2, ph, pw, 3], dict of numpy arrays)."""
    rng = np.random.RandomState(seed)
    scenes = [Scene(scene_w, scene_h, n_objects=4, seed=seed * 1000 + s) for s in range(n_scenes)]
    out = torch.empty((n, 2, patch_h, patch_w, 3), dtype=torch.uint8, device=device)
    sid = rng.randint(0, n_scenes, n)
    x0 = rng.uniform(0, scene_w - patch_w - 2 * max_shift, n) + max_shift
    y0 = rng.uniform(0, scene_h - patch_h - 2 * max_shift, n) + max_shift
    shift = rng.uniform(-max_shift, max_shift, (n, 2))
    t = rng.randint(0, 60, n)
    resp_i = _responses(rng, n, cast)
    resp_j = _responses(rng, n, cast)
    u = torch.arange(patch_w, dtype=torch.float32, device=device)
    v = torch.arange(patch_h, dtype=torch.float32, device=device)
    V, U = torch.meshgrid(v, u, indexing="ij")
    for s in range(n_scenes):
        idx_all = np.nonzero(sid == s)[0]
        for c0 in range(0, idx_all.size, chunk):
            idx = idx_all[c0:c0 + chunk]
            if idx.size == 0:
                continue
            bx = torch.tensor(x0[idx], dtype=torch.float32, device=device).view(-1, 1, 1)
            by = torch.tensor(y0[idx], dtype=torch.float32, device=device).view(-1, 1, 1)
            sx = torch.tensor(shift[idx, 0], dtype=torch.float32, device=device).view(-1, 1, 1)
            sy = torch.tensor(shift[idx, 1], dtype=torch.float32, device=device).view(-1, 1, 1)
            ti = int(np.median(t[idx]))
            Xi, Yi = U + bx, V + by
            rgb_i = scenes[s].render(Xi, Yi, ti)
            rgb_j = scenes[s].render(Xi + sx, Yi + sy, ti)
            sel = lambda r: tuple(a[idx] for a in r)   # noqa: E731
            ii = torch.as_tensor(idx, device=device)
            out[ii, 0] = apply_response(rgb_i, *sel(resp_i))
            out[ii, 1] = apply_response(rgb_j, *sel(resp_j))
    params = dict(gain_i=resp_i[0], gamma_i=resp_i[1], offset_i=resp_i[2], cast_i=resp_i[3],
                  gain_j=resp_j[0], gamma_j=resp_j[1], offset_j=resp_j[2], cast_j=resp_j[3])
    return out, params


def make_window_pairs(n, patch_w=128, patch_h=96, n_frames=3, seed=0, device="cpu", n_scenes=16, scene_w=1152,
                      scene_h=360, n_times=24, n_objects=6, max_shift=3, cast=0.05, chunk=2048):
    """n seeded pairs shaped like a rig's window-pooled overlap: each side of
    a pair is the same crop of one scene at n_frames consecutive times (moving
    objects), the sub-patches stacked in rows, so that its histograms and
    sums pool the window as the estimator pools a rig's overlap over W
    frames. Side j is the crop moved by an integer shift of up to max_shift
    pixels; each side has its own photometric response (see the module
    docstring). The scenes are rendered once per time step and the pairs cut
    from those renders. Returns (pairs uint8 [n, 2, n_frames * patch_h,
    patch_w, 3], dict of the response parameters)."""
    rng = np.random.RandomState(seed)
    scenes = [Scene(scene_w, scene_h, n_objects=n_objects, seed=seed * 1000 + 500 + s) for s in range(n_scenes)]
    u = torch.arange(scene_w, dtype=torch.float32, device=device)
    v = torch.arange(scene_h, dtype=torch.float32, device=device)
    V, U = torch.meshgrid(v, u, indexing="ij")
    renders = torch.empty((n_scenes, n_times, scene_h, scene_w, 3), dtype=torch.float32, device=device)
    for s in range(n_scenes):
        for t in range(n_times):
            renders[s, t] = scenes[s].render(U, V, t)
    sid = rng.randint(0, n_scenes, n)
    t0 = rng.randint(0, n_times - n_frames + 1, n)
    x0 = rng.randint(max_shift, scene_w - patch_w - max_shift, n)
    y0 = rng.randint(max_shift, scene_h - patch_h - max_shift, n)
    sh = rng.randint(-max_shift, max_shift + 1, (n, 2))
    resp_i = _responses(rng, n, cast)
    resp_j = _responses(rng, n, cast)
    out = torch.empty((n, 2, n_frames * patch_h, patch_w, 3), dtype=torch.uint8, device=device)
    ky = torch.arange(patch_h, device=device).view(1, 1, -1, 1)
    kx = torch.arange(patch_w, device=device).view(1, 1, 1, -1)
    kt = torch.arange(n_frames, device=device).view(1, -1, 1, 1)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        m = c1 - c0
        S_ = torch.as_tensor(sid[c0:c1], device=device).view(-1, 1, 1, 1)
        T_ = torch.as_tensor(t0[c0:c1], device=device).view(-1, 1, 1, 1) + kt
        for side, (dx, dy) in enumerate(((np.zeros(m, np.int64), np.zeros(m, np.int64)), (sh[c0:c1, 0], sh[c0:c1, 1]))):
            Y_ = torch.as_tensor(y0[c0:c1] + dy, device=device).view(-1, 1, 1, 1) + ky
            X_ = torch.as_tensor(x0[c0:c1] + dx, device=device).view(-1, 1, 1, 1) + kx
            rgb = renders[S_, T_, Y_, X_].reshape(m, n_frames * patch_h, patch_w, 3)
            r = resp_i if side == 0 else resp_j
            out[c0:c1, side] = apply_response(rgb, *(a[c0:c1] for a in r))
    params = dict(gain_i=resp_i[0], gamma_i=resp_i[1], offset_i=resp_i[2], cast_i=resp_i[3],
                  gain_j=resp_j[0], gamma_j=resp_j[1], offset_j=resp_j[2], cast_j=resp_j[3])
    return out, params
