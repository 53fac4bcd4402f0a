"""Pins of the oracle's pre-warp, local warping and fusion (section 3.1,
section 3.2, Eq. 15-18) against closed forms: identity and integer shifts
reproduce the input bit for bit, bilinear sampling of a linear ramp is exact,
and constant flows over ramp images give a closed-form fused value."""
import numpy as np
import pytest

import oracle
from oracle.pipeline import OracleStitcher


def _T(tx, ty):
    return np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]])


def _zero_flows(o):
    out = []
    for (x0, x1, y0, y1) in o.geom.bands:
        out.append(np.zeros((y1 - y0, x1 - x0, 2), np.float32))
    return out


def test_identity_reproduces_input_bit_for_bit():
    rng = np.random.RandomState(0)
    base = rng.randint(0, 256, (60, 320, 3)).astype(np.uint8)
    frames = [base[:, 0:200].copy(), base[:, 120:320].copy()]
    o = OracleStitcher([_T(0, 0), _T(120, 0)], [200, 200], [60, 60], 320, 60,
                       flags=oracle.BALANCE_OFF, max_flow=4)
    z = _zero_flows(o)
    planes, near, _ = o.frame(frames, z, z)
    assert np.array_equal(planes.transpose(1, 2, 0), base)


def test_integer_translation_is_exact_shift():
    rng = np.random.RandomState(1)
    a = rng.randint(0, 256, (50, 100, 3)).astype(np.uint8)
    b = rng.randint(0, 256, (50, 100, 3)).astype(np.uint8)
    o = OracleStitcher([_T(7, 3), _T(90, 3)], [100, 100], [50, 50], 200, 60,
                       flags=oracle.BALANCE_OFF, max_flow=2)
    assert o.geom.bands == [(90, 107, 3, 53)]
    z = _zero_flows(o)
    planes, _, _ = o.frame([a, b], z, z)
    out = planes.transpose(1, 2, 0)
    assert np.array_equal(out[3:53, 7:90], a[:, 0:83])        # camera a's own columns
    assert np.array_equal(out[3:53, 107:190], b[:, 17:100])   # camera b's own columns
    assert (out[0:3] == 0).all() and (out[53:] == 0).all()    # uncovered rows
    assert (out[:, 0:7] == 0).all() and (out[:, 190:] == 0).all()


def _ramp(w, h, x_off, y_scale=2, y_off=5):
    u = np.arange(w)[None, :].repeat(h, 0)
    v = np.arange(h)[:, None].repeat(w, 1)
    img = np.stack([u + x_off, y_scale * v + y_off, np.full((h, w), 50)], 2)
    assert img.max() <= 255
    return img.astype(np.uint8)


def test_bilinear_of_linear_ramp_is_exact():
    frame = _ramp(200, 60, 10)
    o = OracleStitcher([_T(0.25, 0.375), _T(150.25, 0.375)], [200, 200], [60, 60], 360, 61,
                       flags=oracle.BALANCE_OFF, max_flow=2)
    z = _zero_flows(o)
    _, _, vals = o.frame([frame, frame], z, z)
    ys, xs = np.mgrid[1:59, 2:140]
    v = vals[ys, xs]
    assert np.allclose(v[..., 0], xs - 0.25 + 10, atol=1e-12)
    assert np.allclose(v[..., 1], 2 * (ys - 0.375) + 5, atol=1e-12)
    assert np.allclose(v[..., 2], 50, atol=1e-12)


@pytest.mark.parametrize("printed", [False, True])
def test_constant_flow_closed_form(printed):
    # Pano content: channel 0 = x + 10, channel 1 = 2 y + 5 in both cameras.
    a = _ramp(120, 80, 10)
    b = _ramp(120, 80, 70)
    flags = oracle.BALANCE_OFF | (oracle.FLOW_WEIGHTS_PRINTED if printed else 0)
    o = OracleStitcher([_T(0, 0), _T(60, 0)], [120, 120], [80, 80], 180, 80, flags=flags,
                       max_flow=8)
    x0, x1, y0, y1 = o.geom.bands[0]
    assert (x0, x1, y0, y1) == (60, 120, 0, 80)
    fij, fji = (3.0, -2.0), (-4.0, 1.5)
    Fi = np.zeros((y1 - y0, x1 - x0, 2), np.float32)
    Fj = np.zeros_like(Fi)
    Fi[..., 0], Fi[..., 1] = fij
    Fj[..., 0], Fj[..., 1] = fji
    _, _, vals = o.frame([a, b], [Fi], [Fj])
    ys, xs = np.mgrid[10:70, 70:110]             # interior: no clamping into the band
    tb = (xs - x0 + 0.5) / (x1 - x0)
    ta = 1 - tb
    wa, wb = (ta, tb) if printed else (tb, ta)
    Xa, Ya = xs + wa * fij[0], ys + wa * fij[1]
    Xb, Yb = xs + wb * fji[0], ys + wb * fji[1]
    exp0 = ta * (Xa + 10) + tb * (Xb + 10)
    exp1 = ta * (2 * Ya + 5) + tb * (2 * Yb + 5)
    v = vals[ys, xs]
    assert np.allclose(v[..., 0], exp0, atol=1e-10)
    assert np.allclose(v[..., 1], exp1, atol=1e-10)
    assert np.allclose(v[..., 2], 50, atol=1e-10)


def test_flow_clamped_to_max_and_into_band():
    a = _ramp(120, 40, 10)
    b = _ramp(120, 40, 70)
    o = OracleStitcher([_T(0, 0), _T(60, 0)], [120, 120], [40, 40], 180, 40,
                       flags=oracle.BALANCE_OFF, max_flow=2)
    x0, x1, y0, y1 = o.geom.bands[0]
    Fi = np.zeros((y1 - y0, x1 - x0, 2), np.float32)
    Fi[..., 0] = -50.0                       # clamped to -2
    Fj = np.zeros_like(Fi)
    Fj[..., 0] = -50.0
    _, _, vals = o.frame([a, b], [Fi], [Fj])
    y, x = 20, 61
    tb = (x - x0 + 0.5) / (x1 - x0)
    ta = 1 - tb
    Xa = max(x + tb * -2.0, x0)
    Xb = max(x + ta * -2.0, x0)              # pulled back into the band
    assert np.isclose(vals[y, x, 0], ta * (Xa + 10) + tb * (Xb + 10), atol=1e-10)


def test_blend_continuous_at_band_edges_with_flow():
    a = _ramp(120, 80, 10)
    b = _ramp(120, 80, 70)
    o = OracleStitcher([_T(0, 0), _T(60, 0)], [120, 120], [80, 80], 180, 80,
                       flags=oracle.BALANCE_OFF, max_flow=8)
    x0, x1, y0, y1 = o.geom.bands[0]
    Fi = np.full((y1 - y0, x1 - x0, 2), 6.0, np.float32)
    Fj = np.full((y1 - y0, x1 - x0, 2), -6.0, np.float32)
    _, _, v = o.frame([a, b], [Fi], [Fj])
    # the ramp rises by 1 per column; a jump would show as a step of ~6
    assert abs((v[40, x0, 0] - v[40, x0 - 1, 0]) - 1) < 0.1
    assert abs((v[40, x1, 0] - v[40, x1 - 1, 0]) - 1) < 0.1
    o2 = OracleStitcher([_T(0, 0), _T(60, 0)], [120, 120], [80, 80], 180, 80,
                        flags=oracle.BALANCE_OFF | oracle.FLOW_WEIGHTS_PRINTED, max_flow=8)
    _, _, v2 = o2.frame([a, b], [Fi], [Fj])
    assert abs((v2[40, x0, 0] - v2[40, x0 - 1, 0]) - 1) > 4


def test_band_slivers_and_uncovered():
    rng = np.random.RandomState(2)
    a = rng.randint(0, 256, (100, 200, 3)).astype(np.uint8)
    b = rng.randint(0, 256, (100, 200, 3)).astype(np.uint8)
    o = OracleStitcher([_T(0, 10), _T(100, 0)], [200, 200], [100, 100], 300, 112,
                       flags=oracle.BALANCE_OFF, max_flow=2)
    assert o.geom.bands == [(100, 200, 10, 100)]
    z = _zero_flows(o)
    planes, _, _ = o.frame([a, b], z, z)
    out = planes.transpose(1, 2, 0)
    assert np.array_equal(out[5, 150], b[5, 50])          # only b covers
    assert np.array_equal(out[105, 150], a[95, 150])      # only a covers
    assert (out[105, 250] == 0).all()                     # nobody covers
    assert (out[111, 50] == 0).all()


def test_colour_matrix_and_balance_order():
    """Eq. 4 then Eq. 5: v . M, clamp to [0, 255], F, round half to even."""
    from oracle import balance as bal
    rng = np.random.RandomState(3)
    a = rng.randint(0, 256, (30, 100, 3)).astype(np.uint8)
    b = rng.randint(0, 256, (30, 100, 3)).astype(np.uint8)
    o = OracleStitcher([_T(0, 0), _T(80, 0)], [100, 100], [30, 30], 180, 30, max_flow=2)
    M = np.array([[1.3, 0.1, 0.0], [0.0, 0.9, 0.2], [0.05, 0.0, 1.1]])
    o.M_cam = np.stack([M, np.eye(3)])
    o.curve = bal.curve_params(np.array([20.0, 30, 40]), np.array([200.0, 210, 220]), 0.05)
    z = _zero_flows(o)
    planes, _, _ = o.frame([a, b], z, z)
    out = planes.transpose(1, 2, 0)
    v = a[10, 30].astype(np.float64) @ M
    v = np.clip(v, 0, 255)
    exp = [np.rint(bal.apply(np.array([v[c]]), o.curve, c)[0]) for c in range(3)]
    assert list(out[10, 30]) == exp
