"""Optical flow between the pre-warped images of a pair over its blend band
(paper section 3.2: the flow that drives the local warping of Eq. 17-18).

TEST INFRASTRUCTURE ONLY (see the package header): the CUDA path never
imports this module.

The paper computes the flow with a library routine and does not print the
method; this is a coarse-to-fine block matcher, defined here step by step:

1. Luminance of a pre-warped band image (float RGB):
   Y = round-half-even(clamp((R + 2 G + B) / 4, 0, 255)), an integer image.
2. Pyramid: L = 3 levels; level l + 1 is level l averaged over 2 x 2 blocks
   in integers, (a + b + c + d + 2) // 4, the last row / column repeated when
   the size is odd (its size is ceil(h / 2) x ceil(w / 2)).
3. Matching cost of displacement d at pixel q of a level: the sum over the
   7 x 7 window o in [-3, 3]^2 of |Y_a(q + d + o) - Y_b(q + o)|, coordinates
   clamped into the level's image (a = the image that moves, b = the target).
4. Coarsest level: every d in [-R, R]^2 with R = max(1, ceil(max_flow / 4));
   finer levels: every d in 2 d_up + [-1, 1]^2, d_up the displacement chosen
   at pixel (q_x // 2, q_y // 2) of the level above. The smallest cost wins;
   ties go to the smaller |d - d_start|^2 (d_start = 0 at the coarsest level,
   2 d_up below), then the smaller d_y, then the smaller d_x.
5. Sub-pixel, at the finest level, per axis: with the costs c-, c0, c+ of the
   chosen d and its two neighbours on that axis (integers),
   off = (c- - c+) / (2 (c- - 2 c0 + c+)) in float32 when the denominator is
   positive (else 0), clamped to [-0.5, 0.5]; the flow is float32(d) + off.

flow_ij moves the left camera's image onto the right one's (P_i(q + f) ~
P_j(q), a = i, b = j); flow_ji the other way (a = j, b = i)."""
import math

import numpy as np

from .warp import prewarp

LEVELS = 3
WIN = 3


def band_prewarp(frame, geom, k, band):
    """Camera k's pre-warped image over a band (float64 (bh, bw, 3))."""
    x0, x1, y0, y1 = band
    qy, qx = np.meshgrid(np.arange(y0, y1, dtype=np.float64), np.arange(x0, x1, dtype=np.float64), indexing="ij")
    v = prewarp(frame, geom.Hinv[k], geom.w[k], geom.h[k], qx.ravel(), qy.ravel(), clamp=True)
    return v.reshape(y1 - y0, x1 - x0, 3)


def luminance(P):
    """Step 1: integer luminance of a float RGB image."""
    y = (P[..., 0] + 2.0 * P[..., 1] + P[..., 2]) / 4.0
    return np.rint(np.clip(y, 0.0, 255.0)).astype(np.int64)


def downsample(Y):
    """Step 2: one pyramid level down."""
    h, w = Y.shape
    Yp = np.pad(Y, ((0, h % 2), (0, w % 2)), mode="edge")
    s = Yp[0::2, 0::2] + Yp[1::2, 0::2] + Yp[0::2, 1::2] + Yp[1::2, 1::2]
    return (s + 2) // 4


def cost(Ya, Yb, qx, qy, dx, dy):
    """Step 3 at pixels (qx, qy) (int arrays) for displacements (dx, dy)."""
    h, w = Ya.shape
    c = np.zeros(qx.shape, dtype=np.int64)
    for oy in range(-WIN, WIN + 1):
        for ox in range(-WIN, WIN + 1):
            ax = np.clip(qx + dx + ox, 0, w - 1)
            ay = np.clip(qy + dy + oy, 0, h - 1)
            bx = np.clip(qx + ox, 0, w - 1)
            by = np.clip(qy + oy, 0, h - 1)
            c += np.abs(Ya[ay, ax] - Yb[by, bx])
    return c


def match(Ya, Yb, start_x, start_y, radius):
    """Step 4 on one level: the chosen displacement of every pixel."""
    h, w = Ya.shape
    qy, qx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    best = None
    bx = np.zeros((h, w), np.int64)
    by = np.zeros((h, w), np.int64)
    # candidates in the tie-break order: |d - start|^2, then d_y, then d_x
    cand = sorted(((ex, ey) for ey in range(-radius, radius + 1) for ex in range(-radius, radius + 1)),
                  key=lambda e: (e[0] * e[0] + e[1] * e[1], e[1], e[0]))
    for ex, ey in cand:
        dx, dy = start_x + ex, start_y + ey
        c = cost(Ya, Yb, qx, qy, dx, dy)
        if best is None:
            best, bx, by = c, dx.copy(), dy.copy()
        else:
            take = c < best                          # strict: earlier candidates win ties
            best = np.where(take, c, best)
            bx = np.where(take, dx, bx)
            by = np.where(take, dy, by)
    return bx, by


def _subpixel(cm, c0, cp):
    num = np.float32(cm - cp)
    den = np.float32(2) * np.float32(cm - 2 * c0 + cp)
    with np.errstate(divide="ignore", invalid="ignore"):
        off = np.where(den > 0, num / np.where(den > 0, den, np.float32(1)), np.float32(0)).astype(np.float32)
    return np.clip(off, np.float32(-0.5), np.float32(0.5)).astype(np.float32)


def pyramid(P):
    """Steps 1-2: the integer luminance pyramid of a float RGB image, finest
    level first."""
    pyr = [luminance(P)]
    for _ in range(LEVELS - 1):
        pyr.append(downsample(pyr[-1]))
    return pyr


def flow(Pa, Pb, max_flow):
    """Flow (float32 (bh, bw, 2)) moving image a onto image b (steps 1-5)."""
    return flow_from_pyramids(pyramid(Pa), pyramid(Pb), max_flow)


def flow_from_pyramids(pyr_a, pyr_b, max_flow):
    """Steps 3-5 on given luminance pyramids (integer images, finest first)."""
    radius = max(1, int(math.ceil(max_flow / 2 ** (LEVELS - 1))))
    h, w = pyr_a[-1].shape
    dx = np.zeros((h, w), np.int64)
    dy = np.zeros((h, w), np.int64)
    dx, dy = match(pyr_a[-1], pyr_b[-1], dx, dy, radius)
    for lev in range(LEVELS - 2, -1, -1):
        h, w = pyr_a[lev].shape
        qy, qx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
        sx = 2 * dx[qy // 2, qx // 2]
        sy = 2 * dy[qy // 2, qx // 2]
        dx, dy = match(pyr_a[lev], pyr_b[lev], sx, sy, 1)
    Ya, Yb = pyr_a[0], pyr_b[0]
    h, w = Ya.shape
    qy, qx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    c0 = cost(Ya, Yb, qx, qy, dx, dy)
    offx = _subpixel(cost(Ya, Yb, qx, qy, dx - 1, dy), c0, cost(Ya, Yb, qx, qy, dx + 1, dy))
    offy = _subpixel(cost(Ya, Yb, qx, qy, dx, dy - 1), c0, cost(Ya, Yb, qx, qy, dx, dy + 1))
    out = np.empty((h, w, 2), np.float32)
    out[..., 0] = dx.astype(np.float32) + offx
    out[..., 1] = dy.astype(np.float32) + offy
    return out


def pair_flows(frames, geom, max_flow):
    """(flows_ij, flows_ji) of every pair of a frame."""
    fij, fji = [], []
    for p, band in enumerate(geom.bands):
        Pi = band_prewarp(np.asarray(frames[p]), geom, p, band)
        Pj = band_prewarp(np.asarray(frames[p + 1]), geom, p + 1, band)
        fij.append(flow(Pi, Pj, max_flow))
        fji.append(flow(Pj, Pi, max_flow))
    return fij, fji
