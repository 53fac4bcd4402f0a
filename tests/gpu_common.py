"""Shared helpers of the GPU parity tests: run the CUDA path (through the C
ABI) and the FP64 oracle on the same seeded inputs and compare."""
from __future__ import annotations

import numpy as np
import torch

from oracle.pipeline import OracleStitcher
from paper_2308_09209_b300 import build as _build
from paper_2308_09209_b300 import stitch as S
from synth import Scene, render_camera_frames, rig_for_config, smooth_flow

# Acceptance bar for panoramas (uint8): >= 99.99 % of compared pixels within
# one grey level of the FP64 oracle and none off by more than 2, after leaving
# out (and counting) pixels whose float64 source point lies within 1e-3 px of
# a camera's coverage edge, where float32 and float64 may disagree on
# coverage.
FRAC_WITHIN_1 = 0.9999
MAX_ABS = 2
M_REL_TOL = 1e-4


def ensure_built():
    _build.build()


def flows_for(bands, max_flow, seed, t, device="cuda"):
    fij, fji = [], []
    for p, (x0, x1, y0, y1) in enumerate(bands.tolist()):
        fij.append(smooth_flow(y1 - y0, x1 - x0, max_flow, seed=seed * 97 + 2 * p, t=t, device=device).contiguous())
        fji.append(smooth_flow(y1 - y0, x1 - x0, max_flow, seed=seed * 97 + 2 * p + 1, t=t, device=device).contiguous())
    return fij, fji


class Pair:
    """A CUDA stitcher and an oracle stitcher fed the same frames."""

    def __init__(self, name, seed=0, flags=0, frames_override=None, **over):
        ensure_built()
        self.rig, self.seq = rig_for_config(name, seed=seed, **over)
        rig, seq = self.rig, self.seq
        self.seed = seed
        self.scene = Scene(rig.pano_w, rig.pano_h, n_objects=seq.get("objects", 0), seed=seed)
        ex = rig.extra or {}
        self.proj = dict(projection=ex.get("projection", 0), cyl=ex.get("cyl"))
        self.cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                            max_flow=seq["max_flow"], flags=flags, **self.proj)
        self.st = S.Stitcher(self.cfg)
        self.oracle = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                                     max_flow=seq["max_flow"], flags=flags, **self.proj)

    def inputs(self, t):
        frames = render_camera_frames(self.rig, self.scene, t, device="cuda")
        fij, fji = flows_for(self.st.bands, self.seq["max_flow"], self.seed, t)
        return frames, fij, fji

    def step(self, t, compare_pano=True):
        frames, fij, fji = self.inputs(t)
        self.st.estimate_color(frames)
        pano = self.st.frame(frames, fij, fji)
        torch.cuda.synchronize()
        fr_np = [f.cpu().numpy() for f in frames]
        self.oracle.estimate_color(fr_np)
        out = dict(frames=frames, fij=fij, fji=fji, pano=pano, fr_np=fr_np)
        if compare_pano:
            planes, near, vals = self.oracle.frame(fr_np, [f.cpu().numpy() for f in fij],
                                                   [f.cpu().numpy() for f in fji])
            out.update(planes=planes, near=near)
        return out


def compare_pano(gpu_pano, planes, near, pano_w):
    g = gpu_pano.cpu().numpy()
    assert (g[:, :, pano_w:] == 0).all(), "row padding must be zero"
    g = g[:, :, :pano_w].astype(np.int16)
    o = planes.astype(np.int16)
    d = np.abs(g - o).max(0)
    keep = ~near
    n = int(keep.sum())
    within1 = float((d[keep] <= 1).sum()) / max(n, 1)
    return dict(max=int(d[keep].max()) if n else 0, within1=within1, exact=float((d[keep] == 0).sum()) / max(n, 1),
                n_near=int(near.sum()), n=n)


def assert_pano_ok(rep):
    assert rep["max"] <= MAX_ABS, rep
    assert rep["within1"] >= FRAC_WITHIN_1, rep


def compare_stats(st_gpu, stats_or, n_pairs):
    assert np.array_equal(st_gpu["pooled"].astype(np.int64), stats_or["pooled"])
    for p in range(n_pairs):
        po = stats_or["pairs"][p]
        assert np.array_equal(st_gpu["Hi"][p].astype(np.int64), po["Hi"]), f"Hi pair {p}"
        assert np.array_equal(st_gpu["Hj"][p].astype(np.int64), po["Hj"]), f"Hj pair {p}"
        pix = po["pix_i"].astype(np.int64)
        k = 0
        for c in range(3):
            for d in range(3):
                if c == d:
                    continue
                W = np.bincount(pix[:, d], weights=pix[:, c].astype(np.float64), minlength=256).astype(np.int64)
                assert np.array_equal(st_gpu["Wv"][p][k].astype(np.int64), W), f"W pair {p} ({c},{d})"
                k += 1
        assert np.array_equal(st_gpu["A"][p].astype(np.int64), po["A"]), f"A pair {p}"
        assert np.array_equal(st_gpu["B"][p].astype(np.int64), po["B"]), f"B pair {p}"


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# --------------------------------------------------------------------------- #
# The oracle's whole panorama on every host core (large frames): the colour
# state comes from the caller's oracle; strips of rows are rendered by spawned
# worker processes reading the frame from memory-mapped files.
# --------------------------------------------------------------------------- #
_PW = {}


def _pw_init(rig_args):
    import os
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle.geometry import Geometry
    _PW["geom"] = Geometry(*rig_args[0], projection=rig_args[1], cyl=rig_args[2])


def _pw_rows(task):
    import os
    from oracle.warp import fuse_pixels, finish
    d, n_cams, M_cam, curve, max_flow, flags, r0, r1, W = task
    frames = [np.load(os.path.join(d, f"f{k}.npy"), mmap_mode="r") for k in range(n_cams)]
    fij = [np.load(os.path.join(d, f"a{p}.npy"), mmap_mode="r") for p in range(n_cams - 1)]
    fji = [np.load(os.path.join(d, f"b{p}.npy"), mmap_mode="r") for p in range(n_cams - 1)]
    ys, xs = np.meshgrid(np.arange(r0, r1), np.arange(W), indexing="ij")
    v, c, e = fuse_pixels(frames, _PW["geom"], fij, fji, M_cam, max_flow, flags, xs.ravel(), ys.ravel())
    return r0, finish(v, c, curve, flags), e


def oracle_frame_parallel(pr, fr_np, fij_np, fji_np):
    """(planes (3, H, W) uint8, near-edge mask (H, W)) of the oracle's whole
    panorama for the frame whose colour pr.oracle estimated last."""
    import multiprocessing as mp
    import os
    import tempfile
    rig, o = pr.rig, pr.oracle
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    H, W = rig.pano_h, rig.pano_w
    step = max(1, H // (4 * n))
    rig_args = ((rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h), pr.proj["projection"], pr.proj["cyl"])
    planes = np.zeros((3, H, W), dtype=np.uint8)
    near = np.zeros((H, W), dtype=bool)
    with tempfile.TemporaryDirectory(dir="/dev/shm" if os.path.isdir("/dev/shm") else None) as d:
        for k, f in enumerate(fr_np):
            np.save(os.path.join(d, f"f{k}.npy"), f)
        for p, (a, b) in enumerate(zip(fij_np, fji_np)):
            np.save(os.path.join(d, f"a{p}.npy"), a)
            np.save(os.path.join(d, f"b{p}.npy"), b)
        tasks = [(d, rig.n_cams, o.M_cam, o.curve, o.max_flow, o.flags, r, min(H, r + step), W)
                 for r in range(0, H, step)]
        with mp.get_context("spawn").Pool(n, initializer=_pw_init, initargs=(rig_args,)) as pool:
            for r0, out, e in pool.imap_unordered(_pw_rows, tasks):
                r1 = r0 + out.shape[0] // W
                planes[:, r0:r1] = out.T.reshape(3, r1 - r0, W)
                near[r0:r1] = e.reshape(r1 - r0, W)
    return planes, near
