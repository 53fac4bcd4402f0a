"""Overlap geometry, float64 (paper section 2.1 step 1; section 3.1).

Conventions: pixel centres sit at integer coordinates. A camera homography H
maps camera pixel (u, v, 1) to panorama coordinates (row-vector free, plain
matrix-vector). The panorama pixel q = (x, y) is covered by camera k when its
source point s = H_k^-1 q lies in [0, w_k - 1] x [0, h_k - 1].

The paper computes "the overlap region in the two frames using the
homographic matrix" (section 2.1 step 1) and pre-warps every frame onto the
reference plane (section 3.1). Readings taken here (the paper gives no
formula for the region):

* The blend band of adjacent cameras (a, b = a + 1) is an integer rectangle
  [x0, x1) x [y0, y1) of panorama pixels: columns from the right-most point
  of b's left edge to the left-most point of a's right edge, rows between the
  lowest top edge and the highest bottom edge of the two cameras over those
  columns. Bounds round inward.
* The source rectangle of a band in camera c is the inward-rounded box
  spanned by the band's four corners mapped through H_c^-1.
* Values within 1e-9 of an integer are snapped to it before rounding inward,
  so that float64 noise cannot move an integer bound.

Cylindrical panorama (the large-rig projection): panorama pixel (x, y) is the
ray (sin t, h, cos t) with t = (x - cx) / f and h = (y - cy) / f; camera k's
matrix C_k maps its pixel (u, v, 1) to a ray, and C_k^-1 maps a ray to the
camera's homogeneous pixel. The paper warps onto one reference plane; the
cylinder is the same pre-warp with a different panorama surface. Camera
edges are curves on the cylinder, so the band's columns come from every
pixel of the two edges that bound it, its rows from the coverage of every
band column by both cameras, and a source rectangle from every pixel of the
band's border.
"""
from __future__ import annotations

import math

import numpy as np

SNAP = 1e-9


def ceil_snap(v: float) -> int:
    r = round(v)
    if abs(v - r) < SNAP:
        return int(r)
    return int(math.ceil(v))


def floor_snap(v: float) -> int:
    r = round(v)
    if abs(v - r) < SNAP:
        return int(r)
    return int(math.floor(v))


def invert(H: np.ndarray) -> np.ndarray:
    """Panorama -> camera map: the inverse homography (section 3.1 pre-warp)."""
    return np.linalg.inv(np.asarray(H, dtype=np.float64))


class CylMap:
    """Panorama -> camera map of a cylindrical panorama: A = C_k^-1 applied
    to the ray of panorama point (x, y)."""

    def __init__(self, A, f, cx, cy):
        self.A = np.asarray(A, dtype=np.float64).reshape(3, 3)
        self.f, self.cx, self.cy = float(f), float(cx), float(cy)

    def point(self, x: float, y: float):
        """One point with the C library's sin / cos (the library's host code
        uses the same), term by term in the same order."""
        A = self.A
        th = (x - self.cx) / self.f
        hh = (y - self.cy) / self.f
        d0, d2 = math.sin(th), math.cos(th)
        a = A[0, 0] * d0 + A[0, 1] * hh + A[0, 2] * d2
        b = A[1, 0] * d0 + A[1, 1] * hh + A[1, 2] * d2
        w = A[2, 0] * d0 + A[2, 1] * hh + A[2, 2] * d2
        return a / w, b / w, w

    def map(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        th = (x - self.cx) / self.f
        hh = (y - self.cy) / self.f
        d0, d2 = np.sin(th), np.cos(th)
        A = self.A
        a = A[0, 0] * d0 + A[0, 1] * hh + A[0, 2] * d2
        b = A[1, 0] * d0 + A[1, 1] * hh + A[1, 2] * d2
        w = A[2, 0] * d0 + A[2, 1] * hh + A[2, 2] * d2
        return a / w, b / w, w


class CylCam:
    """Camera -> panorama map of a cylindrical panorama: the ray
    d = C_k (u, v, 1) at azimuth atan2(d_x, d_z) and height
    d_y / sqrt(d_x^2 + d_z^2)."""

    def __init__(self, C, f, cx, cy):
        self.C = np.asarray(C, dtype=np.float64).reshape(3, 3)
        self.f, self.cx, self.cy = float(f), float(cx), float(cy)

    def point(self, u: float, v: float):
        C = self.C
        d0 = C[0, 0] * u + C[0, 1] * v + C[0, 2]
        d1 = C[1, 0] * u + C[1, 1] * v + C[1, 2]
        d2 = C[2, 0] * u + C[2, 1] * v + C[2, 2]
        return self.cx + self.f * math.atan2(d0, d2), self.cy + self.f * (d1 / math.sqrt(d0 * d0 + d2 * d2))

    def map(self, u, v):
        u = np.asarray(u, dtype=np.float64)
        v = np.asarray(v, dtype=np.float64)
        C = self.C
        d0 = C[0, 0] * u + C[0, 1] * v + C[0, 2]
        d1 = C[1, 0] * u + C[1, 1] * v + C[1, 2]
        d2 = C[2, 0] * u + C[2, 1] * v + C[2, 2]
        X = self.cx + self.f * np.arctan2(d0, d2)
        Y = self.cy + self.f * (d1 / np.sqrt(d0 * d0 + d2 * d2))
        return X, Y, np.ones_like(X)


def project(H, x, y):
    """Apply a homography (or a cylinder map) to points (x, y): returns
    (X/W, Y/W, W)."""
    if hasattr(H, "map"):
        return H.map(x, y)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    X = H[0, 0] * x + H[0, 1] * y + H[0, 2]
    Y = H[1, 0] * x + H[1, 1] * y + H[1, 2]
    W = H[2, 0] * x + H[2, 1] * y + H[2, 2]
    return X / W, Y / W, W


def coverage(Hinv, w, h, qx, qy):
    """Is panorama point q inside camera (w, h)? Also the float64 distance of
    its source point to the coverage boundary (used to exclude edge pixels)."""
    sx, sy, sw = project(Hinv, qx, qy)
    inside = (sw > 0) & (sx >= 0) & (sx <= w - 1) & (sy >= 0) & (sy <= h - 1)
    dx = np.minimum(np.abs(sx), np.abs(sx - (w - 1)))
    dy = np.minimum(np.abs(sy), np.abs(sy - (h - 1)))
    near_x = (dx < 1e-3) & (sy >= -1e-3) & (sy <= h - 1 + 1e-3)
    near_y = (dy < 1e-3) & (sx >= -1e-3) & (sx <= w - 1 + 1e-3)
    return inside, near_x | near_y, sx, sy


def camera_corners(H, w, h):
    """Panorama positions of the camera's corner pixel centres TL, TR, BR, BL."""
    u = np.array([0.0, w - 1.0, w - 1.0, 0.0])
    v = np.array([0.0, 0.0, h - 1.0, h - 1.0])
    X, Y, _ = project(np.asarray(H, dtype=np.float64), u, v)
    return np.stack([X, Y], 1)


def _line_y_at(p, q, x):
    """y of the straight line through p and q, at abscissa x."""
    return p[1] + (q[1] - p[1]) * (x - p[0]) / (q[0] - p[0])


def band_rect(Ha, wa, ha, Hb, wb, hb, pano_w, pano_h):
    """Blend band (x0, x1, y0, y1) of the adjacent pair (a left, b right)."""
    ca = camera_corners(Ha, wa, ha)
    cb = camera_corners(Hb, wb, hb)
    TL, TR, BR, BL = 0, 1, 2, 3
    x0 = ceil_snap(max(cb[TL, 0], cb[BL, 0]))
    x1 = floor_snap(min(ca[TR, 0], ca[BR, 0])) + 1
    xl, xr = float(x0), float(x1 - 1)
    tops = [_line_y_at(c[TL], c[TR], xx) for c in (ca, cb) for xx in (xl, xr)]
    bots = [_line_y_at(c[BL], c[BR], xx) for c in (ca, cb) for xx in (xl, xr)]
    y0 = ceil_snap(max(tops))
    y1 = floor_snap(min(bots)) + 1
    x0 = max(x0, 0)
    y0 = max(y0, 0)
    x1 = min(x1, pano_w)
    y1 = min(y1, pano_h)
    return (x0, x1, y0, y1)


def source_rect(Hinv, w, h, band):
    """Source rectangle [rx0, rx1) x [ry0, ry1) of a band inside one camera."""
    x0, x1, y0, y1 = band
    px = np.array([x0, x1 - 1, x1 - 1, x0], dtype=np.float64)
    py = np.array([y0, y0, y1 - 1, y1 - 1], dtype=np.float64)
    sx, sy, _ = project(Hinv, px, py)
    rx0 = ceil_snap(max(sx[0], sx[3]))
    rx1 = floor_snap(min(sx[1], sx[2])) + 1
    ry0 = ceil_snap(max(sy[0], sy[1]))
    ry1 = floor_snap(min(sy[2], sy[3])) + 1
    rx0, ry0 = max(rx0, 0), max(ry0, 0)
    rx1, ry1 = min(rx1, w), min(ry1, h)
    if rx1 <= rx0 or ry1 <= ry0:
        return (0, 0, 0, 0)
    return (rx0, rx1, ry0, ry1)


def _covered_exact(m, w, h, x, y):
    sx, sy, sw = m.point(float(x), float(y))
    return sw > 0 and 0.0 <= sx <= w - 1 and 0.0 <= sy <= h - 1


def band_rect_cyl(ca, ma, wa, ha, cb, mb, wb, hb, pano_w, pano_h):
    """Blend band of a cylindrical pair: columns between the right-most point
    of b's left edge and the left-most point of a's right edge (every edge
    pixel), rows covered by both cameras in every band column. ca / cb map
    camera -> panorama, ma / mb panorama -> camera."""
    xl = max(cb.point(0.0, float(v))[0] for v in range(hb))
    xr = min(ca.point(wa - 1.0, float(v))[0] for v in range(ha))
    x0 = max(ceil_snap(xl), 0)
    x1 = min(floor_snap(xr) + 1, pano_w)
    if x1 - x0 < 2:
        return (x0, x1, 0, 0)
    y0, y1 = 0, pano_h
    ys = np.arange(pano_h, dtype=np.float64)
    for m, w, h in ((ma, wa, ha), (mb, wb, hb)):
        X, Y = np.meshgrid(np.arange(x0, x1, dtype=np.float64), ys)
        sx, sy, sw = m.map(X, Y)
        cov = (sw > 0) & (sx >= 0) & (sx <= w - 1) & (sy >= 0) & (sy <= h - 1)
        # decisions within rounding of the border are taken again with the C library's sin / cos
        near = ((np.minimum(np.abs(sx), np.abs(sx - (w - 1))) < 1e-6) |
                (np.minimum(np.abs(sy), np.abs(sy - (h - 1))) < 1e-6) | (np.abs(sw) < 1e-9))
        for r, c in zip(*np.nonzero(near)):
            cov[r, c] = _covered_exact(m, w, h, X[r, c], Y[r, c])
        for c in range(cov.shape[1]):
            rows = np.nonzero(cov[:, c])[0]
            if rows.size == 0:
                return (x0, x1, 0, 0)
            y0 = max(y0, int(rows[0]))
            y1 = min(y1, int(rows[-1]) + 1)
    return (x0, x1, y0, y1)


def source_rect_cyl(m, w, h, band):
    """Source rectangle of a band in a camera of a cylindrical panorama: the
    inward-rounded box of every pixel of the band's border mapped into it."""
    x0, x1, y0, y1 = band
    l = max(m.point(float(x0), float(y))[0] for y in range(y0, y1))
    r = min(m.point(float(x1 - 1), float(y))[0] for y in range(y0, y1))
    t = max(m.point(float(x), float(y0))[1] for x in range(x0, x1))
    b = min(m.point(float(x), float(y1 - 1))[1] for x in range(x0, x1))
    rx0, rx1 = max(ceil_snap(l), 0), min(floor_snap(r) + 1, w)
    ry0, ry1 = max(ceil_snap(t), 0), min(floor_snap(b) + 1, h)
    if rx1 <= rx0 or ry1 <= ry0:
        return (0, 0, 0, 0)
    return (rx0, rx1, ry0, ry1)


def colour_pairs(n_cams: int, ref: int):
    """Direction of colour transfer per adjacent pair p = (p, p + 1).

    The paper transfers image i onto reference image j (section 2.1 step 3).
    Every pair is oriented toward the reference camera, so chaining the pair
    matrices brings any camera to the reference's colours. Returns a list of
    (i_cam, j_cam) per pair."""
    out = []
    for p in range(n_cams - 1):
        if p + 1 <= ref:
            out.append((p, p + 1))
        else:
            out.append((p + 1, p))
    return out


class Geometry:
    """Everything fixed at initialisation, in float64 / integers."""

    def __init__(self, H, cam_w, cam_h, pano_w, pano_h, ref_cam=None, projection=0, cyl=None):
        self.n = len(cam_w)
        self.w = [int(v) for v in cam_w]
        self.h = [int(v) for v in cam_h]
        self.pano_w = int(pano_w)
        self.pano_h = int(pano_h)
        self.ref = self.n // 2 if ref_cam is None or ref_cam < 0 else int(ref_cam)
        self.projection = int(projection)
        mats = [np.asarray(h, dtype=np.float64).reshape(3, 3) for h in H]
        if self.projection == 0:
            self.H = mats
            self.Hinv = [invert(h) for h in self.H]
        else:
            f, cx, cy = cyl
            self.H = [CylCam(m, f, cx, cy) for m in mats]
            self.Hinv = [CylMap(invert(m), f, cx, cy) for m in mats]
        self.bands = []
        self.rects = []          # per pair: (rect in left camera a, rect in right camera b)
        for p in range(self.n - 1):
            a, b = p, p + 1
            if self.projection == 0:
                band = band_rect(self.H[a], self.w[a], self.h[a], self.H[b], self.w[b], self.h[b],
                                 self.pano_w, self.pano_h)
                rects = (source_rect(self.Hinv[a], self.w[a], self.h[a], band),
                         source_rect(self.Hinv[b], self.w[b], self.h[b], band))
            else:
                band = band_rect_cyl(self.H[a], self.Hinv[a], self.w[a], self.h[a], self.H[b], self.Hinv[b],
                                     self.w[b], self.h[b], self.pano_w, self.pano_h)
                rects = (source_rect_cyl(self.Hinv[a], self.w[a], self.h[a], band),
                         source_rect_cyl(self.Hinv[b], self.w[b], self.h[b], band))
            self.bands.append(band)
            self.rects.append(rects)
        self.pairs = colour_pairs(self.n, self.ref)

    def own_columns(self, k):
        """Columns [lo, hi) of the panorama owned by camera k alone (between bands)."""
        lo = 0 if k == 0 else self.bands[k - 1][1]
        hi = self.pano_w if k == self.n - 1 else self.bands[k][0]
        return lo, hi

    def rect_of(self, p, cam):
        a = p
        return self.rects[p][0] if cam == a else self.rects[p][1]
