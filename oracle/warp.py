"""Pre-warp, optical-flow local warping and weighted-mean fusion, float64
(paper section 3.1, section 3.2, Eq. 15-18).

Per panorama pixel q = (x, y), integer:

* Pre-warp (section 3.1): camera k's value at q is the bilinear sample of
  its frame at s = H_k^-1 q (taps at floor(s) and floor(s) + 1, the far tap
  clamped to the last row / column), defined where q is covered.
* Fusion (Eq. 15): a pixel seen by one camera takes that camera's value; a
  pixel seen by both cameras of a pair takes theta_i P_i + theta_j P_j.
* Local warping (Eq. 17-18), inside a pair's blend band only: image i is
  sampled at X_i = q + theta . flow_ij(q), image j at X_j = q + theta .
  flow_ji(q), where P_k(X) is the bilinear sample of camera k's PRE-WARPED
  image at X (two-stage sampling, as the paper pre-warps first and then
  remaps).

Readings:
* Eq. 16 as printed (a ratio of x-coordinates) does not reach 0 at a band
  edge, so theta is read as a linear ramp across the band's columns:
  theta_j(q) = (x - x0 + 0.5) / (x1 - x0), theta_i = 1 - theta_j, where i is
  the left camera and j the right one.
* Eq. 17 as printed weights flow_ij by theta_i, which makes the output jump
  at the band edge whenever the flow is not zero; the continuous form
  X_i = q + theta_j flow_ij, X_j = q + theta_i flow_ji is the default and the
  printed form is kept behind FLOW_WEIGHTS_PRINTED.
* Flow components are clamped to [-max_flow, max_flow] (IEEE fmin/fmax, so a
  NaN component reads as +max_flow), and X is clamped into the band, which
  lies inside both cameras' coverage, so every remap tap is covered.
* The colour matrix of Eq. 4 is applied to every pixel of a camera (not only
  its overlap), M_k being the camera's matrix chained to the reference.
* Column ownership: camera k alone owns the columns between the band it
  shares with k - 1 and the band it shares with k + 1. There a pixel takes
  camera k's value, else (not covered by k) camera k - 1's, else k + 1's,
  else 0. In a band's columns but outside its rows the pixel blends both
  cameras without flow where both cover it, else takes the one that covers
  it, else 0.
* After fusion each channel is clamped to [0, 255], balanced (Eq. 5, unless
  BALANCE_OFF) and rounded half to even. Uncovered pixels are 0.
"""
from __future__ import annotations

import numpy as np

from . import balance as _bal
from .geometry import project, coverage

BALANCE_OFF = 1
FLOW_WEIGHTS_PRINTED = 4


def _gather(frame, ix, iy):
    return frame[iy, ix].astype(np.float64)


def prewarp(frame, Hinv, w, h, qx, qy, clamp=False):
    """Camera frame bilinearly sampled at s = H^-1 q, float64 (N, 3).

    clamp=True clamps s into the frame first (used inside bands, which the
    geometry guarantees to be covered)."""
    sx, sy, _ = project(Hinv, qx, qy)
    if clamp:
        sx = np.clip(sx, 0.0, w - 1.0)
        sy = np.clip(sy, 0.0, h - 1.0)
    fx0 = np.floor(sx)
    fy0 = np.floor(sy)
    fx = sx - fx0
    fy = sy - fy0
    ix0 = np.clip(fx0, 0, w - 1).astype(np.int64)
    iy0 = np.clip(fy0, 0, h - 1).astype(np.int64)
    ix1 = np.minimum(ix0 + 1, w - 1)
    iy1 = np.minimum(iy0 + 1, h - 1)
    I00 = _gather(frame, ix0, iy0)
    I10 = _gather(frame, ix1, iy0)
    I01 = _gather(frame, ix0, iy1)
    I11 = _gather(frame, ix1, iy1)
    fx = fx[:, None]
    fy = fy[:, None]
    return (1.0 - fy) * ((1.0 - fx) * I00 + fx * I10) + fy * ((1.0 - fx) * I01 + fx * I11)


def remap_sample(frame, Hinv, w, h, band, Xx, Xy):
    """P_k(X): bilinear sample of camera k's pre-warped image at real X (Eq. 18),
    X clamped into the band; the four integer taps are pre-warped values."""
    x0, x1, y0, y1 = band
    Xx = np.clip(Xx, float(x0), float(x1 - 1))
    Xy = np.clip(Xy, float(y0), float(y1 - 1))
    jx = np.floor(Xx)
    jy = np.floor(Xy)
    gx = (Xx - jx)[:, None]
    gy = (Xy - jy)[:, None]
    jx1 = np.minimum(jx + 1, x1 - 1)
    jy1 = np.minimum(jy + 1, y1 - 1)
    P00 = prewarp(frame, Hinv, w, h, jx, jy, clamp=True)
    P10 = prewarp(frame, Hinv, w, h, jx1, jy, clamp=True)
    P01 = prewarp(frame, Hinv, w, h, jx, jy1, clamp=True)
    P11 = prewarp(frame, Hinv, w, h, jx1, jy1, clamp=True)
    return (1.0 - gy) * ((1.0 - gx) * P00 + gx * P10) + gy * ((1.0 - gx) * P01 + gx * P11)


def fuse_pixels(frames, geom, flows_ij, flows_ji, M_cam, max_flow, flags, xs, ys):
    """Fused value (before clamp / balance / rounding) of panorama pixels.

    Returns (val (N, 3) float64, covered (N,) bool, near_edge (N,) bool)."""
    xs = np.asarray(xs, dtype=np.int64)
    ys = np.asarray(ys, dtype=np.int64)
    N = xs.shape[0]
    qx = xs.astype(np.float64)
    qy = ys.astype(np.float64)
    val = np.zeros((N, 3))
    covered = np.zeros(N, dtype=bool)
    near = np.zeros(N, dtype=bool)
    cov = []
    for k in range(geom.n):
        c, e, _, _ = coverage(geom.Hinv[k], geom.w[k], geom.h[k], qx, qy)
        cov.append(c)
        near |= e

    def v_of(k, sel):
        P = prewarp(frames[k], geom.Hinv[k], geom.w[k], geom.h[k], qx[sel], qy[sel])
        return P @ M_cam[k]

    # Columns owned by a single camera.
    for k in range(geom.n):
        lo, hi = geom.own_columns(k)
        own = (xs >= lo) & (xs < hi)
        order = [k] + ([k - 1] if k > 0 else []) + ([k + 1] if k < geom.n - 1 else [])
        todo = own.copy()
        for kk in order:
            sel = todo & cov[kk]
            if sel.any():
                val[sel] = v_of(kk, sel)
                covered[sel] = True
            todo &= ~sel
    # Band columns.
    printed = bool(flags & FLOW_WEIGHTS_PRINTED)
    for p, band in enumerate(geom.bands):
        x0, x1, y0, y1 = band
        a, b = p, p + 1
        cols = (xs >= x0) & (xs < x1)
        if not cols.any():
            continue
        tb = (qx - x0 + 0.5) / float(x1 - x0)      # theta of the right camera b
        ta = 1.0 - tb                               # theta of the left camera a
        inband = cols & (ys >= y0) & (ys < y1)
        if inband.any():
            sel = inband
            fi = np.asarray(flows_ij[p], dtype=np.float64)
            fj = np.asarray(flows_ji[p], dtype=np.float64)
            lx = xs[sel] - x0
            ly = ys[sel] - y0
            fa = np.fmax(np.fmin(fi[ly, lx], max_flow), -max_flow)
            fb = np.fmax(np.fmin(fj[ly, lx], max_flow), -max_flow)
            wa = ta[sel] if printed else tb[sel]
            wb = tb[sel] if printed else ta[sel]
            Xa = qx[sel] + wa * fa[:, 0]
            Ya = qy[sel] + wa * fa[:, 1]
            Xb = qx[sel] + wb * fb[:, 0]
            Yb = qy[sel] + wb * fb[:, 1]
            Pa = remap_sample(frames[a], geom.Hinv[a], geom.w[a], geom.h[a], band, Xa, Ya)
            Pb = remap_sample(frames[b], geom.Hinv[b], geom.w[b], geom.h[b], band, Xb, Yb)
            val[sel] = ta[sel][:, None] * (Pa @ M_cam[a]) + tb[sel][:, None] * (Pb @ M_cam[b])
            covered[sel] = True
        rest = cols & ~inband
        both = rest & cov[a] & cov[b]
        if both.any():
            val[both] = ta[both][:, None] * v_of(a, both) + tb[both][:, None] * v_of(b, both)
            covered[both] = True
        only_a = rest & cov[a] & ~cov[b]
        if only_a.any():
            val[only_a] = v_of(a, only_a)
            covered[only_a] = True
        only_b = rest & cov[b] & ~cov[a]
        if only_b.any():
            val[only_b] = v_of(b, only_b)
            covered[only_b] = True
    return val, covered, near


def finish(val, covered, curve, flags):
    """Clamp to [0, 255], balance (Eq. 5), round half to even; uncovered -> 0."""
    out = np.clip(val, 0.0, 255.0)
    if not (flags & BALANCE_OFF):
        out = np.stack([_bal.apply(out[:, c], curve, c) for c in range(3)], 1)
    out = np.rint(np.clip(out, 0.0, 255.0))
    out[~covered] = 0
    return out.astype(np.uint8)


def stitch(frames, geom, flows_ij, flows_ji, M_cam, curve, max_flow, flags, rows_per_chunk=64, cov_out=None):
    """Whole panorama: (planes (3, H, W) uint8, near_edge (H, W) bool, val (H, W, 3)).
    cov_out (optional (H, W) bool array) receives the covered pixels."""
    W, H = geom.pano_w, geom.pano_h
    planes = np.zeros((3, H, W), dtype=np.uint8)
    near = np.zeros((H, W), dtype=bool)
    vals = np.zeros((H, W, 3))
    xs_row = np.arange(W)
    for r0 in range(0, H, rows_per_chunk):
        r1 = min(H, r0 + rows_per_chunk)
        ys = np.repeat(np.arange(r0, r1), W)
        xs = np.tile(xs_row, r1 - r0)
        v, c, e = fuse_pixels(frames, geom, flows_ij, flows_ji, M_cam, max_flow, flags, xs, ys)
        o = finish(v, c, curve, flags)
        planes[:, r0:r1, :] = o.T.reshape(3, r1 - r0, W)
        near[r0:r1] = e.reshape(r1 - r0, W)
        vals[r0:r1] = v.reshape(r1 - r0, W, 3)
        if cov_out is not None:
            cov_out[r0:r1] = c.reshape(r1 - r0, W)
    return planes, near, vals
