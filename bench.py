#!/usr/bin/env python
"""Throughput benchmark of the stitching hot path on one B300 (or N replicas).

One step = the whole per-frame path (colour statistics, colour estimate,
fused warp / remap / colour / blend / balance) over a batch of F consecutive
synthetic frames of the 4 x 1920x1080 rig, replayed as one CUDA graph through
the C ABI (stitch_sequence). The F frames' inputs (~2.7 GB) are far larger
than the 126 MB L2, so every step streams them from HBM.

Printed JSON line (rank 0): value = whole-job panorama output Mpix/s; e2e =
the same metric through stitch_sequence_host with host buffers (host->device
copies of frames and flows and the device->host copy of the panorama inside
the timed region); roofline = the fused warp stage against the measured HBM
copy bandwidth; cpu_baseline = the FP64 oracle on a bounded sample.

--impl reference times the FP64 oracle on the host cores instead (there is no
other implementation of the paper's method to run).
"""
from __future__ import annotations

import argparse
import faulthandler
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "panorama output Mpix/s & fps (4x1080p), % HBM roofline, batched/learned vs plain"
UNIT = "Mpix/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="4x1920x1080")
    ap.add_argument("--frames", type=int, default=60)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-frames", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# --------------------------------------------------------------------------- #
# distributed plumbing (replicas only: no data-path collective)
# --------------------------------------------------------------------------- #
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if self.pg.get_backend() == "nccl" else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def done(self):
        if self.pg:
            self.pg.destroy_process_group()


# --------------------------------------------------------------------------- #
# workload
# --------------------------------------------------------------------------- #
def make_workload(name, n_frames, seed, device):
    import torch
    from synth import Scene, render_camera_frames, rig_for_config, smooth_flow
    from paper_2308_09209_b300 import stitch as S
    rig, seq = rig_for_config(name, seed=seed)
    cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                   max_flow=seq["max_flow"])
    bands, _ = S.stitch_geometry(cfg)
    scene = Scene(rig.pano_w, rig.pano_h, n_objects=seq["objects"], seed=seed)
    frames, fij, fji = [], [], []
    for t in range(n_frames):
        frames.append(render_camera_frames(rig, scene, t, device=device))
        a, b = [], []
        for p, (x0, x1, y0, y1) in enumerate(bands.tolist()):
            a.append(smooth_flow(y1 - y0, x1 - x0, seq["max_flow"], seed=seed * 97 + 2 * p, t=t,
                                 device=device).contiguous())
            b.append(smooth_flow(y1 - y0, x1 - x0, seq["max_flow"], seed=seed * 97 + 2 * p + 1, t=t,
                                 device=device).contiguous())
        fij.append(a)
        fji.append(b)
    in_bytes = sum(3 * w * h for w, h in zip(rig.cam_w, rig.cam_h))
    flow_bytes = sum(16 * (x1 - x0) * (y1 - y0) for (x0, x1, y0, y1) in bands.tolist())
    out_bytes = 3 * rig.pano_w * rig.pano_h
    return dict(rig=rig, seq=seq, cfg=cfg, bands=bands, frames=frames, fij=fij, fji=fji,
                in_bytes=in_bytes, flow_bytes=flow_bytes, out_bytes=out_bytes,
                pano_px=rig.pano_w * rig.pano_h)


# --------------------------------------------------------------------------- #
# clocks during the timed region
# --------------------------------------------------------------------------- #
class ClockSampler:
    """nvidia-smi samples every 50 ms; stop() keeps those inside [t0, t1]."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            if ts is not None and t0 is not None and not (t0 - 0.06 <= ts <= t1 + 0.06):
                continue
            try:
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- #
# roofline bookkeeping
# --------------------------------------------------------------------------- #
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def traffic_from_profile(workload):
    """dram bytes per fused-warp launch pair from the committed ncu summary, if
    the kernel source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", f"fuse_{workload}.md")
    src = os.path.join(ROOT, "paper_2308_09209_b300", "csrc", "k_fuse.cu")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_frame:\s*([0-9]+)", txt)
    h = re.search(r"k_fuse\.cu sha1:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    if hashlib.sha1(open(src, "rb").read()).hexdigest() != h.group(1):
        return None
    return int(m.group(1))


# --------------------------------------------------------------------------- #
# CPU baseline / reference arm: the FP64 oracle, as it stands
# --------------------------------------------------------------------------- #
def oracle_frames(wl, frame_ids):
    """Run the oracle on the given frames; returns (seconds, output pixels)."""
    import numpy as np
    from oracle.pipeline import OracleStitcher
    rig, seq = wl["rig"], wl["seq"]
    o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                       max_flow=seq["max_flow"])
    host = [([f.cpu().numpy() for f in wl["frames"][t]], [f.cpu().numpy() for f in wl["fij"][t]],
             [f.cpu().numpy() for f in wl["fji"][t]]) for t in frame_ids]
    t0 = time.perf_counter()
    for fr, a, b in host:
        o.estimate_color(fr)
        o.frame(fr, a, b)
    dt = time.perf_counter() - t0
    return dt, len(frame_ids) * wl["pano_px"]


def run_reference(args, dist):
    if dist.rank != 0:
        return
    wl = make_workload(args.workload, max(1, min(args.frames, args.steps + args.warmup)), args.seed, "cpu")
    n = len(wl["frames"])
    times = []
    for s in range(args.warmup + args.steps):
        dt, px = oracle_frames(wl, [s % n])
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = wl["pano_px"] / (ms / 1e3) / 1e6
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one full frame (estimate + fused panorama {wl['rig'].pano_w}x{wl['rig'].pano_h}) per step"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} rig -> {wl['rig'].pano_w}x{wl['rig'].pano_h} planar, "
                                   "FP64 CPU oracle, 1 frame per step",
                       "frames_per_step": 1},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# our CUDA path
# --------------------------------------------------------------------------- #
def run_ours(args, dist):
    ctxs = []
    try:
        _run_ours(args, dist, ctxs)
    finally:
        for st in ctxs:
            st.close()


def _run_ours(args, dist, ctxs):
    import torch
    from paper_2308_09209_b300 import build as _build
    from paper_2308_09209_b300 import stitch as S
    _build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    wl = make_workload(args.workload, args.frames, args.seed + dist.rank, dev)
    F = args.frames
    cfg = wl["cfg"]
    st = S.Stitcher(cfg)
    ctxs.append(st)
    stream = torch.cuda.Stream(device=dev)
    panos = [torch.empty((3, cfg.pano_h, cfg.pitch), dtype=torch.uint8, device=dev) for _ in range(F)]
    frames = [f for fr in wl["frames"] for f in fr]
    fij = [f for fl in wl["fij"] for f in fl]
    fji = [f for fl in wl["fji"] for f in fl]
    torch.cuda.synchronize()

    def step():
        S.stitch_sequence(st.ctx, F, frames, fij, fji, panos, stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    time.sleep(0.2)                      # let the sampler start
    t_begin = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    t_end = time.time()
    dist.barrier()
    clk = clocks.stop(t_begin, t_end)
    ms = e0.elapsed_time(e1) / args.steps
    ms = dist.max(ms)
    rc = S.stitch_sync(st.ctx, stream)
    value = dist.world * F * wl["pano_px"] / (ms / 1e3) / 1e6
    fps = F / (ms / 1e3)

    # Stage durations, live, with CUDA events recorded on the launching stream
    # around each stage (event nodes inside the same graph), same workload.
    S.stitch_profile(st.ctx, True)
    step()
    S.stitch_profile_read(st.ctx)
    acc = dict(stats_ms=0.0, estimate_ms=0.0, fuse_ms=0.0, prewarp_ms=0.0, stats_n=0, estimate_n=0, fuse_n=0,
               prewarp_n=0)
    for _ in range(min(args.steps, 5)):
        step()
        r = S.stitch_profile_read(st.ctx)
        for k in acc:
            acc[k] += r[k]
    S.stitch_profile(st.ctx, False)
    stage_timing = "event nodes in the replayed graph"

    fuse_ms = acc["fuse_ms"] / max(acc["fuse_n"], 1)
    prewarp_ms = acc["prewarp_ms"] / max(acc["prewarp_n"], 1)
    stats_ms = acc["stats_ms"] / max(acc["stats_n"], 1)
    est_ms = acc["estimate_ms"] / max(acc["estimate_n"], 1)
    warp_ms = fuse_ms + prewarp_ms      # the fused warp stage of one frame
    fuse_bytes = wl["in_bytes"] + wl["flow_bytes"] + wl["out_bytes"]
    peak, peak_kind = measured_peaks()
    achieved = fuse_bytes / (warp_ms / 1e3) / 1e9
    traffic = traffic_from_profile(args.workload)
    path_bytes = wl["in_bytes"] + wl["flow_bytes"] + wl["out_bytes"]
    path_gbs = F * path_bytes / (ms / 1e3) / 1e9

    # End to end through host buffers (pinned), same metric.
    n_e2e = min(args.e2e_frames, F)
    st2 = S.Stitcher(cfg)
    ctxs.append(st2)
    h_frames = [f.cpu().pin_memory() for fr in wl["frames"][:n_e2e] for f in fr]
    h_fij = [f.cpu().pin_memory() for fl in wl["fij"][:n_e2e] for f in fl]
    h_fji = [f.cpu().pin_memory() for fl in wl["fji"][:n_e2e] for f in fl]
    h_out = [torch.empty((3, cfg.pano_h, cfg.pitch), dtype=torch.uint8).pin_memory() for _ in range(n_e2e)]
    S.stitch_sequence_host(st2.ctx, n_e2e, h_frames, h_fij, h_fji, h_out, stream)
    dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        S.stitch_sequence_host(st2.ctx, n_e2e, h_frames, h_fij, h_fji, h_out, stream)
    e2e_s = dist.max((time.perf_counter() - t0) / e2e_steps)
    e2e_value = dist.world * n_e2e * wl["pano_px"] / e2e_s / 1e6
    h2d = n_e2e * (wl["in_bytes"] + wl["flow_bytes"])
    d2h = n_e2e * 3 * cfg.pitch * cfg.pano_h

    cpu_baseline = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        dt, px = oracle_frames(wl, [0, 1])
        cpu_baseline = {"value": px / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                        "sample": f"frames 0-1 of the workload: estimate + full {wl['rig'].pano_w}x"
                                  f"{wl['rig'].pano_h} panorama each, numpy float64, one thread"}

    launches = args.steps * F * 4     # stats, estimate, band pre-warp, fuse per frame
    if dist.rank == 0:
        rig = wl["rig"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload} rig (4 cameras 1920x1080 packed RGB) -> "
                                   f"{rig.pano_w}x{rig.pano_h} planar panorama, {F} frames per step, "
                                   f"window {wl['seq']['window']}, max flow {wl['seq']['max_flow']} px",
                       "frames_per_step": F, "fps": fps * dist.world,
                       "l2": "inputs larger than L2 (%.1f GB per step)" % (F * path_bytes / 1e9),
                       "path_bytes_per_frame": path_bytes, "path_hbm_gbs": path_gbs,
                       "path_hbm_frac": path_gbs / peak,
                       "stage_ms_per_frame": {"stats": stats_ms, "estimate": est_ms, "band_prewarp": prewarp_ms,
                                              "fuse": fuse_ms},
                       "stage_timing": stage_timing,
                       "status": rc, "parallelism": f"replicas x{dist.world}"},
            "roofline": {"bound": "hbm", "kernel": "fused warp stage of a frame (k_prewarp_band + k_fuse)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": fuse_bytes},
            "cpu_baseline": cpu_baseline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "frames_per_step": n_e2e},
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)


def main():
    faulthandler.enable()
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        dist.init("gloo")
        try:
            run_reference(args, dist)
        finally:
            dist.done()
        return
    dist.init("nccl")
    try:
        run_ours(args, dist)
    finally:
        dist.done()


if __name__ == "__main__":
    main()
