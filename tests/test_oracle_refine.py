"""Pins of the oracle's homography refinement from the band flows (section
3.1, Eq. 13-14; oracle/refine.py): the median is an order statistic checked
by counting, and known translation / scale errors of the homographies are
undone exactly (translations) or to the stated first order (scales),
including the outward chaining over four cameras."""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle.refine import flow_stats, lower_median, refine


def _T(dx, dy):
    return np.array([[1.0, 0.0, dx], [0.0, 1.0, dy], [0.0, 0.0, 1.0]])


def _rand_H(rng):
    H = np.eye(3) + rng.uniform(-0.02, 0.02, (3, 3))
    H[2] = [rng.uniform(-1e-5, 1e-5), rng.uniform(-1e-5, 1e-5), 1.0]
    H[:2, 2] += rng.uniform(-50, 50, 2)
    return H


def _const_flow(bw, bh, v):
    f = np.empty((bh, bw, 2), np.float32)
    f[..., 0], f[..., 1] = v
    return f


@pytest.mark.parametrize("n", [1, 2, 7, 8, 31, 64])
def test_lower_median_is_the_order_statistic_by_counting(n):
    rng = np.random.default_rng(n)
    v = rng.normal(0, 3, n).astype(np.float32)
    v[rng.integers(0, n, n // 4)] = rng.integers(-3, 3, n // 4)      # ties
    w = np.concatenate([v, np.array([np.nan, np.inf, -np.inf], np.float32)])
    rng.shuffle(w)
    m = lower_median(w)
    k = (n - 1) // 2
    assert m in v
    assert np.sum(v < m) <= k < np.sum(v <= m)
    assert lower_median(np.array([np.nan, np.inf], np.float32)) == 0.0
    assert lower_median(np.zeros(0, np.float32)) == 0.0


def test_forward_differences_are_float32_and_skip_non_finite():
    f = np.zeros((3, 5, 2), np.float32)
    f[..., 0] = np.float32(0.1) * np.arange(5, dtype=np.float32)        # x ramp
    f[..., 1] = (np.float32(0.3) * np.arange(3, dtype=np.float32))[:, None]
    f[1, 2, 0] = np.nan                                                  # kills two x differences
    mx, my, gx, gy = flow_stats(f)
    d = np.diff(f[..., 0], axis=1).astype(np.float32)
    assert gx == lower_median(d) and np.isfinite(gx)
    assert gy == lower_median(np.diff(f[..., 1], axis=0).astype(np.float32))
    assert mx == lower_median(f[..., 0]) and my == np.float32(0.3)


def test_a_translated_left_camera_is_put_back():
    rng = np.random.default_rng(1)
    geom = SimpleNamespace(ref=1, bands=[(500, 640, 0, 360)])
    Ht = [_rand_H(rng), _rand_H(rng)]
    delta = (2.5, -1.25)
    H = [_T(*delta) @ Ht[0], Ht[1]]
    bw, bh = 140, 360
    Hn, prm = refine(geom, H, [_const_flow(bw, bh, delta)], [_const_flow(bw, bh, (-delta[0], -delta[1]))])
    assert tuple(prm[0]) == (-2.5, 1.25, 1.0, 1.0)
    assert np.array_equal(Hn[1], Ht[1])
    assert np.allclose(Hn[0], Ht[0], rtol=0, atol=1e-12 * np.abs(Ht[0]).max())


def test_a_translated_right_camera_is_put_back():
    rng = np.random.default_rng(2)
    geom = SimpleNamespace(ref=0, bands=[(500, 640, 0, 360)])
    Ht = [_rand_H(rng), _rand_H(rng)]
    delta = (-3.0, 0.5)                       # the right content sits displaced by delta against the left
    H = [Ht[0], _T(*delta) @ Ht[1]]
    Hn, prm = refine(geom, H, [_const_flow(140, 360, (-delta[0], -delta[1]))], [_const_flow(140, 360, delta)])
    assert tuple(prm[0]) == (3.0, -0.5, 1.0, 1.0)
    assert np.array_equal(Hn[0], Ht[0])
    assert np.allclose(Hn[1], Ht[1], rtol=0, atol=1e-12 * np.abs(Ht[1]).max())


def test_scale_about_the_band_centre():
    """Left content stretched about the band centre c by 1 + 1/32 in x: the
    flow is (x - c_x) / 32 (exact in float32), the correction scales by
    1 - 1/32 about c and leaves c in place."""
    x0, x1, y0, y1 = 600, 664, 10, 42
    geom = SimpleNamespace(ref=1, bands=[(x0, x1, y0, y1)])
    cx = (x0 + x1 - 1) / 2.0
    xs = np.arange(x0, x1, dtype=np.float64)
    f = np.zeros((y1 - y0, x1 - x0, 2), np.float32)
    f[..., 0] = ((xs - cx) / 32.0).astype(np.float32)[None, :]
    Hn, prm = refine(geom, [np.eye(3), np.eye(3)], [f], [-f])
    assert tuple(prm[0]) == (0.0, 0.0, 1.0 - 1.0 / 32.0, 1.0)
    cy = (y0 + y1 - 1) / 2.0
    A = Hn[0]
    assert np.allclose(A @ [cx, cy, 1.0], [cx, cy, 1.0], rtol=0, atol=1e-12)
    assert np.allclose(A @ [cx + 10.0, cy + 3.0, 1.0], [cx + 10.0 * (1 - 1 / 32), cy + 3.0, 1.0], rtol=0, atol=1e-12)


def test_corrections_chain_outward_from_the_reference():
    """Four cameras, reference 2: camera 0 is off by d0 against camera 1, which
    is off by d1 against the reference; camera 3 is off by d3. The refined
    homographies are the true ones."""
    rng = np.random.default_rng(3)
    geom = SimpleNamespace(ref=2, bands=[(100, 180, 0, 200), (400, 470, 0, 200), (700, 790, 0, 200)])
    Ht = [_rand_H(rng) for _ in range(4)]
    d0, d1, d3 = (1.5, -0.75), (-2.0, 0.25), (0.5, 3.0)
    H = [_T(d0[0] + d1[0], d0[1] + d1[1]) @ Ht[0], _T(*d1) @ Ht[1], Ht[2], _T(*d3) @ Ht[3]]
    neg = lambda v: (-v[0], -v[1])   # noqa: E731
    fij = [_const_flow(80, 200, d0), _const_flow(70, 200, d1), _const_flow(90, 200, neg(d3))]
    fji = [_const_flow(80, 200, neg(d0)), _const_flow(70, 200, neg(d1)), _const_flow(90, 200, d3)]
    Hn, prm = refine(geom, H, fij, fji)
    assert np.array_equal(Hn[2], Ht[2])
    for k in (0, 1, 3):
        assert np.allclose(Hn[k], Ht[k], rtol=0, atol=1e-12 * np.abs(Ht[k]).max()), k
    assert tuple(prm[2]) == (-0.5, -3.0, 1.0, 1.0)


def test_non_finite_flow_samples_are_ignored():
    f = _const_flow(40, 20, (1.25, -0.5))
    g = f.copy()
    g[3, 7] = np.nan
    g[10, :, 1] = np.inf
    assert flow_stats(f) == flow_stats(g)
