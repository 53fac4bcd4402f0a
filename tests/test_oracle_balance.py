"""Pins of the oracle's online colour balancing (section 2.2, Eq. 5-7):
quantile knots against sorting, the 3-frame smoothing against a hand-worked
sequence, and the piecewise curve against its defining properties."""
import os

import numpy as np
import pytest

from oracle import balance as bal

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            out[k] = [float(x) for x in v]
    return out


@pytest.mark.parametrize("seed", range(5))
def test_knots_match_sorted_quantiles(seed):
    rng = np.random.RandomState(seed)
    N = rng.randint(50, 5000)
    vals = np.clip(rng.normal(rng.uniform(60, 200), rng.uniform(5, 80), size=(N, 3)), 0, 255).astype(np.int64)
    hist = np.stack([np.bincount(vals[:, c], minlength=256) for c in range(3)])
    m1, m2 = bal.knots(hist, 0.05)
    for c in range(3):
        s = np.sort(vals[:, c])
        # smallest v whose CDF reaches 5 % (95 %) of N: the ceil(N/20)-th (ceil(19N/20)-th) value
        assert m1[c] == s[-(-N // 20) - 1]
        assert m2[c] == s[-(-19 * N // 20) - 1]


def test_smoothing_hand_worked():
    g = _read_golden("knot_smoothing.txt")
    hist = []
    for t in range(len(g["m1_per_frame"])):
        hist.append((np.full(3, g["m1_per_frame"][t]), np.full(3, g["m2_per_frame"][t])))
        s1, s2 = bal.smooth(hist)
        assert np.allclose(s1, g["m1_smoothed"][t]) and np.allclose(s2, g["m2_smoothed"][t])


def _curve(m1, m2):
    return bal.curve_params(np.full(3, float(m1)), np.full(3, float(m2)), 0.05)


@pytest.mark.parametrize("m1,m2", [(5, 245), (30, 200), (12.75, 242.25), (1, 254), (100, 101.5),
                                   (0.333, 180), (40, 255)])
def test_curve_properties(m1, m2):
    p = _curve(m1, m2)
    x = np.linspace(0, 255, 200001)
    F = bal.apply(x, p, 0)
    assert (np.diff(F) >= -1e-12).all(), "F must be monotone non-decreasing"
    d1, d2 = 255 * 0.05, 255 * 0.95
    if m1 > 0:
        assert abs(bal.apply(np.array([0.0]), p, 0)[0]) < 1e-12
    if m2 < 255:
        assert abs(bal.apply(np.array([255.0]), p, 0)[0] - 255) < 1e-9
    assert abs(bal.apply(np.array([float(m1)]), p, 0)[0] - d1) < 1e-9
    assert abs(bal.apply(np.array([float(m2)]), p, 0)[0] - d2) < 1e-9
    # C1 at both knots: one-sided difference quotients agree with the slope s
    h = 1e-6
    s = (d2 - d1) / (m2 - m1)
    for k in (m1, m2):
        if (k == m1 and m1 > 0) or (k == m2 and m2 < 255):
            left = (bal.apply(np.array([k]), p, 0) - bal.apply(np.array([k - h]), p, 0))[0] / h
            right = (bal.apply(np.array([k + h]), p, 0) - bal.apply(np.array([k]), p, 0))[0] / h
            assert abs(left - s) < 1e-4 * max(1, s) and abs(right - s) < 1e-4 * max(1, s)


def test_identity_when_knots_equal_targets():
    p = _curve(255 * 0.05, 255 * 0.95)
    x = np.linspace(0, 255, 1001)
    assert np.allclose(bal.apply(x, p, 0), x, atol=1e-9)


def test_degenerate_span_is_identity():
    p = _curve(100, 100.5)
    x = np.linspace(0, 255, 101)
    assert np.array_equal(bal.apply(x, p, 0), x)


def test_gamma_tails_closed_form():
    # m1 = 51, m2 = 204: s = 229.5 / 153 = 1.5, g1 = 1.5 * 51 / 12.75 = 6,
    # g2 = 1.5 * 51 / 12.75 = 6; F(25.5) = 12.75 * 0.5^6; F(229.5) = 255 - 12.75 * 0.5^6
    p = _curve(51, 204)
    assert np.isclose(p["s"][0], 1.5) and np.isclose(p["g1"][0], 6) and np.isclose(p["g2"][0], 6)
    assert np.isclose(bal.apply(np.array([25.5]), p, 0)[0], 12.75 / 64)
    assert np.isclose(bal.apply(np.array([229.5]), p, 0)[0], 255 - 12.75 / 64)
    assert np.isclose(bal.apply(np.array([127.5]), p, 0)[0], 12.75 + 1.5 * 76.5)


# --- balance on the stitched image (one-frame lag) ---------------------------

def test_output_histogram_hand_worked():
    """Three pixels worked by hand: v clamped to [0, 255], q = rint(16 v),
    bin = (q + 8) // 16; the uncovered pixel does not count."""
    from oracle.balance import output_histogram
    v = np.array([[0.0, 255.0, 127.5],       # q = 0, 4080, 2040 -> bins 0, 255, 128
                  [127.53, 0.03, 300.0],     # q = 2040, 0, 4080 -> bins 128, 0, 255
                  [-5.0, 64.49, 64.5]])      # not covered
    h = output_histogram(v, np.array([True, True, False]))
    want = np.zeros((3, 256), dtype=np.int64)
    want[0, 0] = want[0, 128] = 1
    want[1, 255] = want[1, 0] = 1
    want[2, 128] = want[2, 255] = 1
    assert np.array_equal(h, want)
    # on the grid of sixteenths: 64.5 -> q 1032 -> bin 65; 64.4375 -> q 1031 -> bin 64;
    # 64.40625 -> 16 v = 1030.5, to even q 1030 -> bin 64
    assert output_histogram(np.array([[64.5, 64.4375, 64.40625]]), np.array([True]))[:, 64:66].tolist() == \
        [[0, 1], [1, 0], [1, 0]]


def test_balance_on_stitched_image_lags_one_frame():
    """Two cameras at integer offsets seeing one mosaic (M = I, zero flow):
    frame 0 is not balanced and its panorama is the mosaic; frame 1's knots
    are the lambda quantiles of that mosaic's histogram, and with a constant
    mosaic the smoothing of Eq. 6-7 keeps them."""
    from oracle.pipeline import OracleStitcher
    from oracle import BALANCE_OUTPUT
    rng = np.random.RandomState(4)
    h, w, off = 40, 60, 40
    mosaic = np.clip(rng.normal(120, 40, (h, off + w, 3)), 0, 255).astype(np.uint8)
    T = lambda tx: np.array([[1.0, 0, tx], [0, 1.0, 0], [0, 0, 1.0]])
    frames = [mosaic[:, :w].copy(), mosaic[:, off:off + w].copy()]
    o = OracleStitcher([T(0), T(off)], [w, w], [h, h], off + w, h, window=3, max_flow=2.0, flags=BALANCE_OUTPUT)
    fl = [np.zeros((h, w - off, 2), np.float32)]
    o.estimate_color(frames)
    assert bool(np.all(o.curve["identity"]))
    planes, near, vals = o.frame(frames, fl, fl)
    assert np.array_equal(planes.transpose(1, 2, 0), mosaic)
    hist = np.stack([np.bincount(mosaic[:, :, c].ravel(), minlength=256) for c in range(3)])
    assert np.array_equal(o.out_hist, hist)
    o.estimate_color(frames)
    m1, m2 = bal.knots(hist, 0.05)
    assert np.array_equal(o.curve["m1"], m1) and np.array_equal(o.curve["m2"], m2)
    o.frame(frames, fl, fl)
    o.estimate_color(frames)
    assert np.array_equal(o.curve["m1"], m1) and np.array_equal(o.curve["m2"], m2)
