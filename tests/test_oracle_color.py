"""Pins of the oracle's 3D-M colour transfer (section 2.1, Eq. 1-4).

Each pin checks the oracle against something other than itself: brute-force
counting, an independent sort-based formulation of histogram specification,
numpy's least-squares solver on the literally stacked (3n x 3) system of
Eq. 2, closed forms (self-transfer, exact gains) and a hand-worked example.
"""
import os

import numpy as np
import pytest

from oracle import color as col
from oracle.pipeline import OracleStitcher

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *vals = line.split()
        out[k] = [float(v) for v in vals]
    return out


def test_histograms_brute_force():
    rng = np.random.RandomState(0)
    pix = rng.randint(0, 256, size=(500, 3)).astype(np.uint8)
    H = col.channel_histograms(pix)
    for c in range(3):
        counts = [0] * 256
        for p in pix[:, c]:
            counts[int(p)] += 1
        assert list(H[c]) == counts
    assert (H.sum(1) == 500).all()


def test_spec_lut_hand_worked_example():
    g = _read_golden("spec_lut_example.txt")
    pi = np.array(g["pixels_i"], dtype=np.int64)
    pj = np.array(g["pixels_j"], dtype=np.int64)
    # channel 0 carries the example; channels 1, 2 are identical on both sides
    Pi = np.stack([pi, pi % 2, pi % 3], 1)
    Pj_other = np.stack([np.zeros_like(pj), pj % 2, pj % 3], 1)
    Hi = col.channel_histograms(Pi)
    Hj = col.channel_histograms(Pj_other)
    Hj[0] = np.bincount(pj, minlength=256)
    lut = col.spec_lut(Hi, Hj)
    assert list(lut[0, :4]) == [int(v) for v in g["lut_0_to_3"]]
    X = pi.astype(np.int64)
    Y = lut[0][X]
    assert int((X * X).sum()) == int(g["A"][0])
    assert int((X * Y).sum()) == int(g["B"][0])


def _spec_by_sorting(vals_i, vals_j):
    """Independent formulation: the level of j at the same quantile rank.
    L(v) = sorted_j[ceil(CDF_i(v) * n_j / n_i) - 1] (exact integer ceil)."""
    si = np.sort(vals_i)
    sj = np.sort(vals_j)
    ni, nj = len(si), len(sj)
    out = np.zeros(256, dtype=np.int64)
    for v in range(256):
        cdf = int(np.searchsorted(si, v, side="right"))
        if cdf == 0:
            out[v] = 0                      # CDF_j(0) * n_i >= 0 always holds
            continue
        k = -(-cdf * nj // ni)              # ceil
        out[v] = sj[k - 1]
    return out


@pytest.mark.parametrize("seed", range(6))
def test_spec_lut_matches_sort_formulation(seed):
    rng = np.random.RandomState(seed)
    ni, nj = rng.randint(5, 400), rng.randint(5, 400)
    pi = rng.randint(rng.randint(0, 60), rng.randint(120, 256), size=(ni, 3))
    pj = np.clip(rng.normal(128, 40, size=(nj, 3)), 0, 255).astype(np.int64)
    lut = col.spec_lut(col.channel_histograms(pi), col.channel_histograms(pj))
    for c in range(3):
        ref = _spec_by_sorting(pi[:, c], pj[:, c])
        occupied = np.bincount(pi[:, c], minlength=256) > 0
        assert (lut[c][occupied] == ref[occupied]).all()
        assert (np.diff(lut[c]) >= 0).all()          # monotone


def test_spec_lut_identity_and_shift():
    rng = np.random.RandomState(3)
    pi = rng.randint(10, 200, size=(1000, 3))
    H = col.channel_histograms(pi)
    lut = col.spec_lut(H, H)
    occ = H > 0
    assert (lut[occ] == np.broadcast_to(np.arange(256), (3, 256))[occ]).all()
    lut2 = col.spec_lut(H, col.channel_histograms(pi + 37))
    assert (lut2[occ] == (np.broadcast_to(np.arange(256), (3, 256)) + 37)[occ]).all()


def _stacked_lstsq(frames_i, luts):
    """Eq. 2 literally: stack I_Ti, I_(T-1)i, ... into a (3n x 3) system."""
    Ii = np.vstack([f.astype(np.float64) for f in frames_i])
    Ij = np.vstack([np.stack([l[c][f[:, c]] for c in range(3)], 1).astype(np.float64)
                    for f, l in zip(frames_i, luts)])
    return np.linalg.lstsq(Ii, Ij, rcond=None)[0]


@pytest.mark.parametrize("seed", range(4))
def test_window_M_matches_stacked_least_squares(seed):
    rng = np.random.RandomState(seed)
    frames_i, frames_j, luts = [], [], []
    A = np.zeros((3, 3), dtype=np.int64)
    B = np.zeros((3, 3), dtype=np.int64)
    for t in range(3):
        pi = rng.randint(0, 256, size=(300, 3))
        pj = np.clip(pi * rng.uniform(0.7, 1.3, 3) + rng.normal(0, 6, (300, 3)), 0, 255).astype(np.int64)
        lut = col.spec_lut(col.channel_histograms(pi), col.channel_histograms(pj))
        a, b = col.normal_equations(pi, lut)
        A += a
        B += b
        frames_i.append(pi)
        luts.append(lut)
    M, ok = col.solve_transfer(A, B)
    assert ok
    M_ref = _stacked_lstsq(frames_i, luts)
    assert np.allclose(M, M_ref, rtol=1e-9, atol=1e-11)


def test_self_transfer_gives_identity():
    rng = np.random.RandomState(1)
    pi = rng.randint(0, 256, size=(2000, 3))
    H = col.channel_histograms(pi)
    lut = col.spec_lut(H, H)
    A, B = col.normal_equations(pi, lut)
    assert (A == B).all()
    M, ok = col.solve_transfer(A, B)
    assert ok and np.allclose(M, np.eye(3), atol=1e-12)


def test_exact_gain_gives_diagonal_M():
    # Image j = 2 * image i exactly (no clipping): the specification maps v to
    # 2v, so B = 2A and M = 2 I.
    rng = np.random.RandomState(2)
    pi = rng.randint(0, 128, size=(5000, 3))
    lut = col.spec_lut(col.channel_histograms(pi), col.channel_histograms(2 * pi))
    A, B = col.normal_equations(pi, lut)
    assert (B == 2 * A).all()
    M, ok = col.solve_transfer(A, B)
    assert ok and np.allclose(M, 2 * np.eye(3), atol=1e-12)


def test_value_weighted_histograms_reproduce_B():
    """B_cd = sum_v L_d(v) W_cd(v) with W_cd(v) = sum of channel c over the
    pixels whose channel d equals v (the one-pass form the GPU uses), checked
    against the direct B of Eq. 3 computed by the oracle."""
    rng = np.random.RandomState(4)
    pi = rng.randint(0, 256, size=(3000, 3))
    pj = rng.randint(20, 240, size=(2500, 3))
    lut = col.spec_lut(col.channel_histograms(pi), col.channel_histograms(pj))
    _, B = col.normal_equations(pi, lut)
    for c in range(3):
        for d in range(3):
            W = np.zeros(256, dtype=np.int64)
            for p in range(pi.shape[0]):
                W[pi[p, d]] += pi[p, c]
            assert int((lut[d] * W).sum()) == int(B[c, d])


def test_flat_overlap_is_singular():
    pi = np.tile(np.array([[40, 90, 160]]), (1000, 1))
    lut = col.spec_lut(col.channel_histograms(pi), col.channel_histograms(pi))
    A, B = col.normal_equations(pi, lut)
    M, ok = col.solve_transfer(A, B)
    assert not ok and M is None


def test_chain_to_reference():
    rng = np.random.RandomState(5)
    Ms = [np.eye(3) + 0.1 * rng.randn(3, 3) for _ in range(3)]
    from oracle.geometry import colour_pairs
    pairs = colour_pairs(4, 2)
    C = col.chain_to_reference(Ms, pairs, 2, 4)
    assert np.allclose(C[2], np.eye(3))
    assert np.allclose(C[1], Ms[1])
    assert np.allclose(C[0], Ms[0] @ Ms[1])
    assert np.allclose(C[3], Ms[2])
    # Row-vector convention (Eq. 4): v . M_0 == (v . M_(0->1)) . M_(1->2)
    v = rng.rand(3)
    assert np.allclose(v @ C[0], (v @ Ms[0]) @ Ms[1])


def test_pipeline_keeps_previous_M_when_singular():
    # Two cameras side by side with an integer offset; frame 0 has texture,
    # frame 1 is flat in the overlap -> M of frame 1 = M of frame 0 with a
    # window of 1 (2D-M).
    T = lambda tx: np.array([[1.0, 0, tx], [0, 1.0, 0], [0, 0, 1.0]])
    o = OracleStitcher([T(0), T(60)], [100, 100], [50, 50], 160, 50, window=1)
    rng = np.random.RandomState(0)
    f0 = [rng.randint(0, 256, (50, 100, 3)).astype(np.uint8) for _ in range(2)]
    assert o.estimate_color(f0)
    M0 = o.M_pair[0].copy()
    flat = [np.full((50, 100, 3), 77, np.uint8) for _ in range(2)]
    assert not o.estimate_color(flat)
    assert np.array_equal(o.M_pair[0], M0)


def test_pipeline_recovers_known_gain_on_rig():
    """A camera that is the reference scene times a per-channel gain g (no
    gamma, offset or clipping) gets M close to diag(1 / g) from the whole
    estimate chain (geometry, histograms, specification, window solve)."""
    import torch
    from synth import make_rig, Scene, render_camera_frames
    rig = make_rig([320, 320], [180, 180], overlap=(0.3, 0.3), rot_deg=2.0, photometric=False,
                   seed=11)
    sc = Scene(rig.pano_w, rig.pano_h, seed=11)
    fr = [np.rint(0.75 * f.numpy()).astype(np.uint8)
          for f in render_camera_frames(rig, sc, 0, photometric=False)]
    g = np.array([0.8, 1.1, 0.9])
    fr[0] = np.rint(fr[0].astype(np.float64) * g).astype(np.uint8)
    assert fr[0].max() < 255 and fr[1].max() < 255
    o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=3)
    for _ in range(3):
        assert o.estimate_color(fr)
    M = o.M_cam[0]
    assert np.allclose(np.diag(M), 1 / g, rtol=0.03)
    assert np.abs(M - np.diag(np.diag(M))).max() < 0.03
    assert np.array_equal(o.M_cam[1], np.eye(3))
