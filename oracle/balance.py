"""Online colour balancing with a piecewise function, float64 (section 2.2, Eq. 5-7).

The paper splits every channel's levels into dark [0, m1], normal [m1, m2]
and bright [m2, 255] ranges, balancing the normal range linearly
(F(x) = a + b x) and the two tails with gamma curves (F(x) = a + T (x/T)^b)
(Eq. 5). m1 and m2 are the levels holding lambda and (1 - lambda) of the
channel histogram, lambda = 0.05, and both knots are averaged over the
current and the last two frames (Eq. 6-7), with the first two frames using
the frames that exist.

Readings (the paper gives no formula for the curve's targets or exponents):
* lambda = 0.05 is a fraction of the pixels (5 %). It is kept as an integer
  count of millionths, lambda_q = round(lambda * 1e6), so the quantile is
  exact: m1 = smallest v with 1e6 * CDF(v) >= lambda_q * N, m2 likewise with
  (1e6 - lambda_q) * N.
* The histogram is the pooled full-frame histogram of all raw camera frames
  of the current frame index.
* Targets: an equalised histogram puts its lambda-quantiles at d1 = 255 lambda
  and d2 = 255 (1 - lambda). Linear part F = d1 + s (x - m1) with
  s = (d2 - d1) / (m2 - m1); dark tail F = d1 (x / m1)^g1; bright tail
  F = 255 - (255 - d2) ((255 - x) / (255 - m2))^g2; exponents g1 = s m1 / d1
  and g2 = s (255 - m2) / (255 - d2) make F continuous with a continuous
  slope at both knots.
* If m2 - m1 < 1 the curve is the identity. With m1 = 0 the dark tail is
  empty, with m2 = 255 the bright tail is empty.

Balance on the stitched image (flag BALANCE_OUTPUT, the other reading of
"the whole stitched image"): the knots of frame T come from the histogram of
the stitched panorama of frame T - 1 before its balance (a one-frame lag),
over its covered pixels. Readings:
* The histogram is of the fused, clamped value v before Eq. 5 (the balanced
  output's quantiles sit at the targets, so feeding it back would make every
  other frame's curve the identity).
* A pixel's bin is its value on the output table's grid of sixteenths,
  rounded: q = round_half_even(16 v), bin = floor((q + 8) / 16).
* Frame 0 has no stitched predecessor: its curve is the identity; Eq. 6-7
  average the knots of the frames that have one (at most the last three).
"""

from __future__ import annotations

import numpy as np

SMOOTH_FRAMES = 3          # Eq. 6-7: current frame and its last two


def lambda_q(lam: float) -> int:
    return int(round(lam * 1e6))


def knots(pooled_hist: np.ndarray, lam: float):
    """Per-channel integer knots (m1, m2) from a (3, 256) histogram."""
    lq = lambda_q(lam)
    m1 = np.zeros(3, dtype=np.int64)
    m2 = np.zeros(3, dtype=np.int64)
    for c in range(3):
        h = np.asarray(pooled_hist[c], dtype=np.int64)
        N = int(h.sum())
        cdf = np.cumsum(h)
        lo = lq * N
        hi = (1000000 - lq) * N
        m1[c] = next(v for v in range(256) if 1000000 * int(cdf[v]) >= lo)
        m2[c] = next(v for v in range(256) if 1000000 * int(cdf[v]) >= hi)
    return m1, m2


def smooth(history):
    """Eq. 6-7: mean of the knots of the current frame and up to two earlier
    ones. ``history`` lists (m1, m2) per frame, oldest first."""
    recent = history[-SMOOTH_FRAMES:]
    m1 = sum(np.asarray(h[0], dtype=np.float64) for h in recent) / len(recent)
    m2 = sum(np.asarray(h[1], dtype=np.float64) for h in recent) / len(recent)
    return m1, m2


def curve_params(m1, m2, lam: float):
    """Per-channel parameters of F (dictionary of float64 arrays)."""
    lam = lambda_q(lam) / 1e6
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    d1 = 255.0 * lam
    d2 = 255.0 * (1.0 - lam)
    ident = (m2 - m1) < 1.0
    span = np.where(ident, 1.0, m2 - m1)
    s = (d2 - d1) / span
    g1 = s * m1 / d1
    g2 = s * (255.0 - m2) / (255.0 - d2)
    return dict(m1=m1, m2=m2, d1=np.full(3, d1), d2=np.full(3, d2), s=s, g1=g1, g2=g2,
                identity=ident)


def apply(x, params, c: int):
    """F_c(x) for channel c, x already clamped to [0, 255] (Eq. 5)."""
    x = np.asarray(x, dtype=np.float64)
    if params["identity"][c]:
        return x.copy()
    m1, m2 = params["m1"][c], params["m2"][c]
    d1, d2 = params["d1"][c], params["d2"][c]
    s, g1, g2 = params["s"][c], params["g1"][c], params["g2"][c]
    out = d1 + s * (x - m1)
    with np.errstate(all="ignore"):
        if m1 > 0:
            dark = x < m1
            out = np.where(dark, d1 * np.power(np.maximum(x, 0.0) / m1, g1), out)
        if m2 < 255:
            bright = x > m2
            out = np.where(bright, 255.0 - (255.0 - d2) * np.power(np.maximum(255.0 - x, 0.0) / (255.0 - m2), g2), out)
    return out


def output_histogram(vals, covered):
    """(3, 256) int64 histogram of a stitched panorama before its balance:
    per covered pixel and channel, the fused value v clamped to [0, 255], put
    on the grid of sixteenths q = round_half_even(16 v) and binned at
    floor((q + 8) / 16)."""
    v = np.clip(np.asarray(vals, dtype=np.float64).reshape(-1, 3), 0.0, 255.0)
    cov = np.asarray(covered, dtype=bool).reshape(-1)
    q = np.rint(16.0 * v[cov]).astype(np.int64)
    b = (q + 8) // 16
    out = np.zeros((3, 256), dtype=np.int64)
    for c in range(3):
        for x in b[:, c]:
            out[c, x] += 1
    return out
