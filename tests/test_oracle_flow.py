"""Pins of the oracle's band optical flow (section 3.2; oracle/flow.py): the
luminance rounding and the pyramid step by hand, the block matcher against a
per-pixel brute force written with plain loops (ties included), the
sub-pixel parabola in closed form, and known translations recovered."""
import numpy as np
import pytest

from oracle.flow import WIN, _subpixel, downsample, flow, luminance, match


def test_luminance_rounds_half_to_even_and_clamps():
    P = np.array([[[1, 0, 0], [2, 0, 0], [6, 0, 0], [0, 1, 0], [300, 300, 300], [-5, 0, 0]]], np.float64)
    assert luminance(P).tolist() == [[0, 0, 2, 0, 255, 0]]      # 0.25, 0.5, 1.5, 0.5, 300, -1.25


def test_downsample_by_hand():
    Y = np.array([[0, 4, 8], [12, 16, 20], [24, 28, 32]], np.int64)
    # edge-padded to 4 x 4: blocks (0,4,12,16) (8,8,20,20) (24,28,24,28) (32,32,32,32)
    assert downsample(Y).tolist() == [[8, 14], [26, 32]]
    assert downsample(np.full((5, 7), 9, np.int64)).tolist() == np.full((3, 4), 9).tolist()


def _brute(Ya, Yb, sx, sy, radius):
    h, w = Ya.shape
    bx = np.zeros((h, w), np.int64)
    by = np.zeros((h, w), np.int64)
    for y in range(h):
        for x in range(w):
            best = None
            for ey in range(-radius, radius + 1):
                for ex in range(-radius, radius + 1):
                    dx, dy = sx[y, x] + ex, sy[y, x] + ey
                    c = 0
                    for oy in range(-WIN, WIN + 1):
                        for ox in range(-WIN, WIN + 1):
                            a = Ya[min(max(y + dy + oy, 0), h - 1), min(max(x + dx + ox, 0), w - 1)]
                            b = Yb[min(max(y + oy, 0), h - 1), min(max(x + ox, 0), w - 1)]
                            c += abs(int(a) - int(b))
                    key = (c, ex * ex + ey * ey, ey, ex)
                    if best is None or key < best[0]:
                        best = (key, dx, dy)
            bx[y, x], by[y, x] = best[1], best[2]
    return bx, by


@pytest.mark.parametrize("levels,radius", [(2, 2), (4, 1)])
def test_matcher_equals_brute_force(levels, radius):
    rng = np.random.default_rng(levels)
    Ya = rng.integers(0, levels, (9, 11))           # few levels: many ties
    Yb = rng.integers(0, levels, (9, 11))
    sx = rng.integers(-1, 2, (9, 11))
    sy = rng.integers(-1, 2, (9, 11))
    got = match(Ya, Yb, sx, sy, radius)
    want = _brute(Ya, Yb, sx, sy, radius)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_subpixel_closed_form():
    cm = np.array([10, 100, 0, 3, 7, 3])
    c0 = np.array([2, 0, 0, 9, 7, 5])
    cp = np.array([6, 0, 0, 5, 7, 9])
    off = _subpixel(cm, c0, cp)
    assert off.dtype == np.float32
    assert off[0] == np.float32(4) / np.float32(24)     # (10 - 6) / (2 (10 - 4 + 6))
    assert off[1] == np.float32(0.5)                    # 100 / 200
    assert off[2] == 0 and off[3] == 0 and off[4] == 0  # flat or concave: no fit
    assert off[5] == np.float32(-0.5)                   # (3 - 9) / (2 (3 - 10 + 9)) = -1.5, clamped


def test_constant_images_give_zero_flow():
    P = np.full((20, 30, 3), 77.0)
    f = flow(P, P, 8.0)
    assert f.dtype == np.float32 and np.all(f == 0)


def _smooth_texture(rng, h, w):
    n = rng.uniform(0, 1, (h, w, 3))
    k = np.ones(7) / 7
    for _ in range(2):
        n = np.apply_along_axis(lambda r: np.convolve(r, k, mode="same"), 0, n)
        n = np.apply_along_axis(lambda r: np.convolve(r, k, mode="same"), 1, n)
    return 255.0 * (n - n.min()) / (n.max() - n.min())


@pytest.mark.parametrize("t", [(3, -2), (-5, 1), (0, 4), (7, -6)])
def test_integer_translation_is_found(t):
    """b(q) = a(q + t) for a seeded smooth random texture: away from the
    borders the flow is t to within the sub-pixel step at 99 % or more of the
    pixels (a 7 x 7 window still meets the aperture problem now and then),
    and wherever the integer part is t its cost is zero."""
    rng = np.random.default_rng(7)
    big = _smooth_texture(rng, 140, 170)
    h, w, m = 112, 144, 12
    Pa = big[m:m + h, m:m + w]
    Pb = big[m + t[1]:m + t[1] + h, m + t[0]:m + t[0] + w]
    f = flow(Pa, Pb, 8.0)
    inner = f[24:-24, 24:-24]
    ok = (np.abs(inner[..., 0] - t[0]) <= 0.5) & (np.abs(inner[..., 1] - t[1]) <= 0.5)
    assert ok.mean() >= 0.99, ok.mean()
    assert np.all(np.abs(f) <= 8 + 4 + 2 + 1 + 0.5)    # reach of the search: 4 R + 2 + 1, plus the sub-pixel step
