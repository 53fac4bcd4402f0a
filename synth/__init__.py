"""Seeded synthetic inputs for the video-stitching hot path.

This package draws inputs and nothing else: camera rigs (ground-truth and
coarse camera->panorama homographies), a procedural scene, per-camera
photometric distortions, moving objects and smooth flow fields. It holds none
of the stitching method's arithmetic (no warping, histograms, colour transfer,
balance or blending), so both the FP64 oracle tests and the CUDA path can
consume its output without sharing any of the method's code.

All randomness is drawn on the host from ``numpy.random.RandomState(seed)``;
per-pixel rendering runs in float32 torch on whichever device is asked for.
Rendering on CPU and on CUDA may differ by one grey level in a few pixels,
which does not matter: every test hands the SAME uint8 tensors to both sides.

Workload recipe (the paper's own video database is private, so these stand in
for it): a scene that is a sum of 64 Gaussian colour blobs plus 4-octave value
noise, optional translating textured rectangles as moving objects; cameras
placed left to right with a given horizontal overlap and a random in-plane
rotation of up to +-3 degrees; per-camera, per-channel gain U(0.8, 1.2), gamma
U(0.9, 1.1) and offset U(-8, 8), optionally a 3x3 colour cast; flow fields
that are sums of low-frequency plane waves limited to the overlap bands;
and, for the learned estimator, pairs of patches of the same content under
two independent photometric responses.
"""
from .rig import Rig, make_rig, rig_for_config, CONFIGS, BATCH_RIGS
from .scene import Scene, render_camera_frames
from .flow import smooth_flow
from .pairs import make_pairs, make_window_pairs, apply_response

__all__ = ["Rig", "make_rig", "rig_for_config", "CONFIGS", "BATCH_RIGS", "Scene",
           "render_camera_frames", "smooth_flow", "make_pairs", "make_window_pairs", "apply_response"]
