"""Camera rigs: ground-truth and coarse camera->panorama homographies.

A rig places cameras left to right on the panorama plane. Camera k's
ground-truth map G_k takes a camera pixel (u, v) (pixel centres at integers)
to panorama coordinates: rotate by theta_k about the image centre, then move
the centre to (cx_k, cy). The coarse homography H_k handed to the stitcher is
G_k composed with a small random perturbation (the paper's "coarse camera
calibration" whose error the optical flow absorbs). The perturbation keeps
the misalignment within a few pixels, below the configured maximum flow.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Rig:
    n_cams: int
    cam_w: list
    cam_h: list
    G: np.ndarray            # (n, 3, 3) ground truth, camera -> panorama
    H: np.ndarray            # (n, 3, 3) coarse, camera -> panorama (stitcher input)
    pano_w: int
    pano_h: int
    gain: np.ndarray         # (n, 3)
    gamma: np.ndarray        # (n, 3)
    offset: np.ndarray       # (n, 3)
    cast: np.ndarray         # (n, 3, 3), identity unless a colour cast is asked for
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_pairs(self) -> int:
        return self.n_cams - 1


def _translate(tx, ty):
    return np.array([[1.0, 0.0, tx], [0.0, 1.0, ty], [0.0, 0.0, 1.0]])


def _rotate(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def make_rig(cam_w, cam_h, overlap=(0.2, 0.2), rot_deg=3.0, perturb=0.0,
             pano_w=None, pano_h=None, cast_offdiag=0.0, photometric=True,
             seed=0) -> Rig:
    """Draw a rig of len(cam_w) cameras.

    overlap: (lo, hi) fraction of the narrower camera's width shared by each
    adjacent pair, drawn uniformly; ignored when pano_w is given (cameras are
    then spaced evenly so the rig spans exactly pano_w columns).
    perturb: size of the coarse-calibration error (0.01 = the configs' 1%):
    linear entries move by up to 0.2*perturb, the translation by up to
    250*perturb pixels.
    """
    rng = np.random.RandomState(seed)
    n = len(cam_w)
    cam_w = [int(w) for w in cam_w]
    cam_h = [int(h) for h in cam_h]
    ph = int(pano_h) if pano_h is not None else max(cam_h)
    cx = np.zeros(n)
    cx[0] = (cam_w[0] - 1) / 2.0
    if pano_w is not None and n > 1:
        span = pano_w - (cam_w[0] - 1) / 2.0 - (cam_w[-1] - 1) / 2.0 - 1.0
        for k in range(1, n):
            cx[k] = cx[0] + span * k / (n - 1)
    else:
        for k in range(1, n):
            o = rng.uniform(overlap[0], overlap[1])
            shared = o * min(cam_w[k - 1], cam_w[k])
            cx[k] = cx[k - 1] + cam_w[k - 1] / 2.0 + cam_w[k] / 2.0 - shared
    pw = int(pano_w) if pano_w is not None else int(math.ceil(cx[-1] + cam_w[-1] / 2.0))
    cy = (ph - 1) / 2.0
    theta = np.deg2rad(rng.uniform(-rot_deg, rot_deg, size=n))
    G = np.zeros((n, 3, 3))
    H = np.zeros((n, 3, 3))
    for k in range(n):
        c_img = ((cam_w[k] - 1) / 2.0, (cam_h[k] - 1) / 2.0)
        G[k] = _translate(cx[k], cy) @ _rotate(theta[k]) @ _translate(-c_img[0], -c_img[1])
        if perturb > 0:
            a, b, c, d = rng.uniform(-0.2 * perturb, 0.2 * perturb, size=4)
            tx, ty = rng.uniform(-250 * perturb, 250 * perturb, size=2)
            P = np.array([[1 + a, b, tx], [c, 1 + d, ty], [0.0, 0.0, 1.0]])
            P = _translate(*c_img) @ P @ _translate(-c_img[0], -c_img[1])
            H[k] = G[k] @ P
        else:
            H[k] = G[k].copy()
    if photometric:
        gain = rng.uniform(0.8, 1.2, size=(n, 3))
        gamma = rng.uniform(0.9, 1.1, size=(n, 3))
        offset = rng.uniform(-8.0, 8.0, size=(n, 3))
    else:
        gain = np.ones((n, 3))
        gamma = np.ones((n, 3))
        offset = np.zeros((n, 3))
    cast = np.tile(np.eye(3), (n, 1, 1))
    if cast_offdiag > 0:
        for k in range(n):
            off = rng.uniform(-cast_offdiag, cast_offdiag, size=(3, 3))
            np.fill_diagonal(off, 0.0)
            cast[k] = np.eye(3) + off
    return Rig(n, cam_w, cam_h, G, H, pw, ph, gain, gamma, offset, cast, seed)


def _rx(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _ry(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _rz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def make_cyl_rig(cam_w, cam_h, f_cam, overlap=0.2, f_pano=None, pano_h=None, pitch_deg=1.0, roll_deg=1.0,
                 yaw_jitter_deg=0.3, perturb_deg=0.0, cast_offdiag=0.0, photometric=True, seed=0) -> Rig:
    """A rotating rig on a cylindrical panorama. Camera k (focal f_cam, pixel
    centre in the image middle) looks at azimuth psi_k; successive azimuths
    are (1 - overlap) of a camera's horizontal field of view apart, plus a
    small jitter, with small random pitch and roll. G_k / H_k are the true /
    coarse maps from camera pixel (u, v, 1) to a viewing ray, R_k^T K^-1; the
    coarse one adds a random rotation of up to perturb_deg degrees. The
    panorama (f_pano pixels per radian, default f_cam) spans the rig's
    azimuth range; rig.extra holds projection = 1 and cyl = (f, cx, cy)."""
    rng = np.random.RandomState(seed)
    n = len(cam_w)
    cam_w = [int(w) for w in cam_w]
    cam_h = [int(h) for h in cam_h]
    fov = 2.0 * math.atan((max(cam_w) / 2.0) / f_cam)
    step = (1.0 - overlap) * fov
    psi = np.array([(k - (n - 1) / 2.0) * step for k in range(n)])
    psi += np.deg2rad(rng.uniform(-yaw_jitter_deg, yaw_jitter_deg, n))
    pitch = np.deg2rad(rng.uniform(-pitch_deg, pitch_deg, n))
    roll = np.deg2rad(rng.uniform(-roll_deg, roll_deg, n))
    f = float(f_pano if f_pano is not None else f_cam)
    lo = psi[0] - fov / 2.0
    hi = psi[-1] + fov / 2.0
    pw = int(math.ceil(f * (hi - lo)))
    ph = int(pano_h) if pano_h is not None else max(cam_h)
    cx = -f * lo
    cy = (ph - 1) / 2.0
    G = np.zeros((n, 3, 3))
    H = np.zeros((n, 3, 3))
    for k in range(n):
        K = np.array([[f_cam, 0.0, (cam_w[k] - 1) / 2.0], [0.0, f_cam, (cam_h[k] - 1) / 2.0], [0.0, 0.0, 1.0]])
        R = _rz(roll[k]) @ _rx(pitch[k]) @ _ry(psi[k]).T          # world -> camera
        G[k] = R.T @ np.linalg.inv(K)
        if perturb_deg > 0:
            a, b, c = np.deg2rad(rng.uniform(-perturb_deg, perturb_deg, 3))
            H[k] = (_rz(c) @ _rx(b) @ _ry(a) @ R).T @ np.linalg.inv(K)
        else:
            H[k] = G[k].copy()
    if photometric:
        gain = rng.uniform(0.8, 1.2, size=(n, 3))
        gamma = rng.uniform(0.9, 1.1, size=(n, 3))
        offset = rng.uniform(-8.0, 8.0, size=(n, 3))
    else:
        gain, gamma, offset = np.ones((n, 3)), np.ones((n, 3)), np.zeros((n, 3))
    cast = np.tile(np.eye(3), (n, 1, 1))
    if cast_offdiag > 0:
        for k in range(n):
            off = rng.uniform(-cast_offdiag, cast_offdiag, size=(3, 3))
            np.fill_diagonal(off, 0.0)
            cast[k] = np.eye(3) + off
    return Rig(n, cam_w, cam_h, G, H, pw, ph, gain, gamma, offset, cast, seed,
               extra=dict(projection=1, cyl=(f, cx, cy)))


# The workloads, by what they are. Each entry gives the rig recipe plus the
# per-sequence parameters (frames, temporal window, maximum flow, objects).
CONFIGS = {
    "2x640x360": dict(cams=[(640, 360)] * 2, pano_w=1150, pano_h=360, overlap=(0.2, 0.2),
                      perturb=0.0, frames=8, window=3, max_flow=3.0, objects=0),
    "4x1920x1080": dict(cams=[(1920, 1080)] * 4, pano_w=None, pano_h=1080, overlap=(0.15, 0.25),
                        perturb=0.01, frames=60, window=5, max_flow=8.0, objects=6),
    "6x1920x1080": dict(cams=[(1920, 1080)] * 6, pano_w=None, pano_h=1080, overlap=(0.15, 0.25),
                        perturb=0.01, frames=8, window=3, max_flow=3.0, objects=0),
    "2x1280x720": dict(cams=[(1280, 720)] * 2, pano_w=None, pano_h=720, overlap=(0.15, 0.25),
                       perturb=0.01, frames=8, window=3, max_flow=3.0, objects=0),
    "3x1920x1080": dict(cams=[(1920, 1080)] * 3, pano_w=None, pano_h=1080, overlap=(0.15, 0.25),
                        perturb=0.01, frames=8, window=3, max_flow=3.0, objects=0),
    "4x3840x2160": dict(cams=[(3840, 2160)] * 4, pano_w=None, pano_h=2160, overlap=(0.15, 0.25),
                        perturb=0.01, frames=8, window=3, max_flow=3.0, objects=0),
    # one rig mixing resolutions: six 1080p cameras followed by two 720p cameras
    "6x1920x1080+2x1280x720": dict(cams=[(1920, 1080)] * 6 + [(1280, 720)] * 2, pano_w=None, pano_h=1080,
                                   overlap=(0.15, 0.25), perturb=0.01, frames=8, window=3, max_flow=3.0,
                                   objects=0),
}

# Cylindrical rigs (rotating cameras on a cylindrical panorama).
CONFIGS["8x3840x2160cyl"] = dict(cams=[(3840, 2160)] * 8, projection=1, f_cam=4117.0, overlap=0.2, perturb_deg=0.2,
                                 frames=120, window=7, max_flow=16.0, objects=12)
CONFIGS["4x640x360cyl"] = dict(cams=[(640, 360)] * 4, projection=1, f_cam=686.0, overlap=0.2, perturb_deg=0.0,
                               frames=8, window=3, max_flow=3.0, objects=0)

# The batched workload: four independent rigs of uneven geometry stitched together.
BATCH_RIGS = ("6x1920x1080+2x1280x720", "3x1920x1080", "4x3840x2160", "2x1280x720")


def rig_for_config(name: str, seed: int = 0, **over) -> tuple[Rig, dict]:
    """Return (rig, sequence parameters) for a named workload."""
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    ws = [c[0] for c in cfg["cams"]]
    hs = [c[1] for c in cfg["cams"]]
    if cfg.get("projection", 0) == 1:
        rig = make_cyl_rig(ws, hs, cfg["f_cam"], overlap=cfg.get("overlap", 0.2), f_pano=cfg.get("f_pano"),
                           pano_h=cfg.get("pano_h"), perturb_deg=cfg.get("perturb_deg", 0.0),
                           cast_offdiag=cfg.get("cast_offdiag", 0.0), seed=seed)
        return rig, cfg
    rig = make_rig(ws, hs, overlap=cfg["overlap"], rot_deg=cfg.get("rot_deg", 3.0),
                   perturb=cfg["perturb"], pano_w=cfg["pano_w"], pano_h=cfg["pano_h"],
                   cast_offdiag=cfg.get("cast_offdiag", 0.0), seed=seed)
    return rig, cfg
