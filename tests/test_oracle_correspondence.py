"""Pins of the oracle's one-frame colour transfer from pixel correspondences
(the 2D-M comparison of Tables 2-3; oracle/correspondence.py): the normal
equations recover an exact linear map, agree with a QR least-squares solve
of the stacked system on noisy data, and give the identity for a camera
against itself; the band sums are the sums over the band's pre-warped
samples."""
import numpy as np

from oracle.correspondence import pair_M, pair_sums, solve
from oracle.flow import band_prewarp
from oracle.geometry import Geometry
from synth import Scene, render_camera_frames, rig_for_config


def test_exact_linear_map_is_recovered():
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 255, (500, 3))
    M0 = np.eye(3) + rng.uniform(-0.1, 0.1, (3, 3))
    M = solve(X.T @ X, X.T @ (X @ M0))
    assert np.allclose(M, M0, rtol=0, atol=1e-12)


def test_matches_qr_least_squares_on_noisy_data():
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 255, (2000, 3))
    Y = X @ (np.eye(3) * 1.1) + rng.normal(0, 3, (2000, 3))
    M = solve(X.T @ X, X.T @ Y)
    M_qr = np.linalg.lstsq(X, Y, rcond=None)[0]
    assert np.allclose(M, M_qr, rtol=0, atol=1e-10)


def test_rig_sums_and_self_map():
    rig, seq = rig_for_config("2x640x360", seed=2)
    geom = Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h)
    frames = [f.numpy() for f in render_camera_frames(rig, Scene(rig.pano_w, rig.pano_h, seed=2), 0)]
    A, B = pair_sums(frames, geom, 0)
    i, j = geom.pairs[0]
    X = band_prewarp(frames[i], geom, i, geom.bands[0]).reshape(-1, 3)
    Y = band_prewarp(frames[j], geom, j, geom.bands[0]).reshape(-1, 3)
    assert np.allclose(A, np.einsum("nc,nd->cd", X, X), rtol=1e-12)
    assert np.allclose(B, np.einsum("nc,nd->cd", X, Y), rtol=1e-12)
    # the source camera against itself (Y = X): the identity
    M = solve(A, A)
    assert np.allclose(M, np.eye(3), rtol=0, atol=1e-12)
    Mp = pair_M(frames, geom)
    assert Mp.shape == (1, 3, 3) and np.allclose(Mp[0], solve(A, B))
