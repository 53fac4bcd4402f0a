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

# numpy's bundled OpenBLAS reads this when numpy is first imported (bench.py
# imports numpy lazily): the oracle's timings are of one host core.
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

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
    ap.add_argument("--e2e-frames", type=int, default=16)
    ap.add_argument("--tile-shape", type=int, default=-1, choices=[-1, 0, 1, 2, 3],
                    help="fuse tile shape index (-1: the library's autotuner picks it)")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="reference arm: seconds of oracle work for all warm-up and timed steps together")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / learned / cylindrical comparisons (rank 0 of a 1-GPU run only)")
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
def make_workload(name, n_frames, seed, device, library=True):
    """Seeded frames and flows of a workload. library=False (the oracle
    timings) takes the band sizes from the oracle's own geometry and never
    loads the CUDA library."""
    import numpy as np
    from synth import Scene, render_camera_frames, rig_for_config, smooth_flow
    rig, seq = rig_for_config(name, seed=seed)
    ex = rig.extra or {}
    if library:
        from paper_2308_09209_b300 import stitch as S
        cfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                       max_flow=seq["max_flow"], projection=ex.get("projection", 0), cyl=ex.get("cyl"))
        bands, _ = S.stitch_geometry(cfg)
    else:
        from oracle.geometry import Geometry
        cfg = None
        g = Geometry(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, projection=ex.get("projection", 0),
                     cyl=ex.get("cyl"))
        bands = np.asarray(g.bands, dtype=np.int64)
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


def issue_from_profiles(workload):
    """Warp instructions per frame of the whole path (k_stats, k_estimate,
    k_prewarp_band, k_fuse, k_fuse_band, k_fuse_own) from the committed ncu
    summaries of one capture, if none of their sources changed since (else
    None), with the fuse tile shape (w, h) the capture ran."""
    names = ("fuse", "stats", "estimate")
    paths = [os.path.join(ROOT, "profiles", f"{n}_{workload}.md") for n in names]
    if not all(os.path.exists(p) for p in paths):
        return None
    txt = open(paths[0]).read()
    m = re.search(r"## k_fuse_own<(\d+), (\d+)>", txt)
    if not m:
        return None
    shas = dict(re.findall(r"(k_\w+\.cu) sha1:\s*([0-9a-f]+)", txt))
    for src in ("k_fuse.cu", "k_stats.cu", "k_estimate.cu"):
        f = os.path.join(ROOT, "paper_2308_09209_b300", "csrc", src)
        if shas.get(src) != hashlib.sha1(open(f, "rb").read()).hexdigest():
            return None
    total = 0.0
    for p in paths:
        vals = re.findall(r"warp instructions \(`smsp__inst_executed\.sum`\) \| ([0-9.]+) inst", open(p).read())
        if not vals:
            return None
        total += sum(float(v) for v in vals)
    return total, (int(m.group(1)), int(m.group(2)))


# --------------------------------------------------------------------------- #
# CPU baseline / reference arm: the FP64 oracle, as it stands
# --------------------------------------------------------------------------- #
def host_link_gbs(dev, stream, mib=256, reps=5):
    """Pinned host <-> device copy bandwidth of one large cudaMemcpyAsync per
    direction (CUDA events on the copying stream), the bound of any
    host-buffer path."""
    import torch
    h = torch.empty(mib << 20, dtype=torch.uint8).pin_memory()
    d = torch.empty(mib << 20, dtype=torch.uint8, device=dev)
    out = {}
    with torch.cuda.stream(stream):
        for name, fn in (("h2d_gbs", lambda: d.copy_(h, non_blocking=True)),
                         ("d2h_gbs", lambda: h.copy_(d, non_blocking=True))):
            fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            out[name] = reps * (mib << 20) / (e0.elapsed_time(e1) / 1e3) / 1e9
    del h, d
    return out


def one_thread():
    """Context that holds numpy's BLAS / OpenMP pools to one thread, so that
    the oracle's timing is that of one host core (threadpoolctl when it is
    installed; otherwise OPENBLAS_NUM_THREADS, set above, does it)."""
    import contextlib
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        return contextlib.nullcontext()
    return threadpool_limits(limits=1)


def oracle_frames(wl, frame_ids, keep=False, flags=0):
    """Run the oracle on the given frames; returns (seconds, output pixels,
    [(planes, near-edge mask)] when keep, process CPU seconds)."""
    from oracle.pipeline import OracleStitcher
    rig, seq = wl["rig"], wl["seq"]
    ex = rig.extra or {}
    o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                       max_flow=seq["max_flow"], projection=ex.get("projection", 0), cyl=ex.get("cyl"), flags=flags)
    host = [([f.cpu().numpy() for f in wl["frames"][t]], [f.cpu().numpy() for f in wl["fij"][t]],
             [f.cpu().numpy() for f in wl["fji"][t]]) for t in frame_ids]
    outs = []
    with one_thread():
        c0 = time.process_time()
        t0 = time.perf_counter()
        for fr, a, b in host:
            o.estimate_color(fr)
            planes, near, _ = o.frame(fr, a, b)
            if keep:
                outs.append((planes, near))
        dt = time.perf_counter() - t0
        cpu = time.process_time() - c0
    return dt, len(frame_ids) * wl["pano_px"], outs, cpu


def oracle_check_rigs(items, n_samples=40000):
    """Frame 0 of each batched rig against the oracle on sampled pixels (half
    of them in the blend bands)."""
    import numpy as np
    from oracle.pipeline import OracleStitcher
    res = []
    rng = np.random.default_rng(0)
    for it in items:
        rig, seq = it["rig"], it["seq"]
        o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                           max_flow=seq["max_flow"], flags=it["flags"])
        o.estimate_color(it["frames"])
        xs = rng.integers(0, rig.pano_w, n_samples)
        ys = rng.integers(0, rig.pano_h, n_samples)
        for i in range(n_samples // 2):
            x0, x1, y0, y1 = o.geom.bands[i % len(o.geom.bands)]
            xs[i], ys[i] = rng.integers(x0, x1), rng.integers(y0, y1)
        vals, near = o.pixels(it["frames"], it["fij"], it["fji"], xs, ys)
        d = np.abs(it["pano"][:, ys, xs].T.astype(np.int16) - vals.astype(np.int16)).max(1)[~near]
        res.append({"rig": "x".join(map(str, (len(rig.cam_w), rig.pano_w, rig.pano_h))), "max_abs": int(d.max()),
                    "frac_within_1": float((d <= 1).mean()), "frac_exact": float((d == 0).mean()),
                    "samples": int(d.size)})
    return res


def oracle_error(gpu_panos, oracle_outs, pano_w):
    """Per-output error of the GPU panoramas against the FP64 oracle's (grey
    levels, pixels within 1e-3 px of a coverage edge left out and counted)."""
    import numpy as np
    mx, n, n1, n0, nn = 0, 0, 0, 0, 0
    for g, (planes, near) in zip(gpu_panos, oracle_outs):
        d = np.abs(g.cpu().numpy()[:, :, :pano_w].astype(np.int16) - planes.astype(np.int16)).max(0)[~near]
        mx = max(mx, int(d.max()) if d.size else 0)
        n += d.size
        n1 += int((d <= 1).sum())
        n0 += int((d == 0).sum())
        nn += int(near.sum())
    return {"max_abs": mx, "frac_within_1": n1 / max(n, 1), "frac_exact": n0 / max(n, 1), "n_near_edge": nn,
            "frames": len(gpu_panos)}


def host_info():
    """Cores this process may run on, and the CPU model."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": n, "cpu_model": model}


_MC = {}


def _mc_init(rig_args):
    # one per worker process: the oracle's geometry of the rig
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle.geometry import Geometry
    _MC["geom"] = Geometry(*rig_args[0], projection=rig_args[1], cyl=rig_args[2])


def _mc_rows(task):
    # one strip of rows of one frame: the oracle's fused pixels through the balance
    import numpy as np
    from oracle.warp import fuse_pixels, finish
    d, M_cam, curve, max_flow, flags, r0, r1, W = task
    n_cams = len(_MC["geom"].w)
    frames = [np.load(os.path.join(d, f"f{k}.npy"), mmap_mode="r") for k in range(n_cams)]
    fij = [np.load(os.path.join(d, f"a{p}.npy"), mmap_mode="r") for p in range(n_cams - 1)]
    fji = [np.load(os.path.join(d, f"b{p}.npy"), mmap_mode="r") for p in range(n_cams - 1)]
    ys, xs = np.meshgrid(np.arange(r0, r1), np.arange(W), indexing="ij")
    v, c, _ = fuse_pixels(frames, _MC["geom"], fij, fji, M_cam, max_flow, flags, xs.ravel(), ys.ravel())
    return r0, finish(v, c, curve, flags)


def oracle_all_cores(wl, frame_ids, flags=0):
    """The oracle on every host core: per frame the colour estimate (serial,
    in this process) and the fused panorama in strips of rows over a pool of
    spawned worker processes reading the frame from memory-mapped files.
    Returns (seconds, output pixels, workers); the files are written outside
    the timed region."""
    import multiprocessing as mp
    import tempfile
    import numpy as np
    from oracle.pipeline import OracleStitcher
    rig, seq = wl["rig"], wl["seq"]
    ex = rig.extra or {}
    o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                       max_flow=seq["max_flow"], projection=ex.get("projection", 0), cyl=ex.get("cyl"), flags=flags)
    n = host_info()["nproc"]
    H, W = rig.pano_h, rig.pano_w
    step = max(1, H // (4 * n))
    rig_args = ((rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h), ex.get("projection", 0), ex.get("cyl"))
    dt = 0.0
    with tempfile.TemporaryDirectory(dir="/dev/shm" if os.path.isdir("/dev/shm") else None) as d, \
            mp.get_context("spawn").Pool(n, initializer=_mc_init, initargs=(rig_args,)) as pool:
        pool.map(_mc_init, [rig_args] * n)          # every worker started and warm
        for t in frame_ids:
            fr = [f.cpu().numpy() for f in wl["frames"][t]]
            for k, f in enumerate(fr):
                np.save(os.path.join(d, f"f{k}.npy"), f)
            for p, (a, b) in enumerate(zip(wl["fij"][t], wl["fji"][t])):
                np.save(os.path.join(d, f"a{p}.npy"), a.cpu().numpy())
                np.save(os.path.join(d, f"b{p}.npy"), b.cpu().numpy())
            t0 = time.perf_counter()
            with one_thread():
                o.estimate_color(fr)
            tasks = [(d, o.M_cam, o.curve, o.max_flow, flags, r, min(H, r + step), W) for r in range(0, H, step)]
            pool.map(_mc_rows, tasks)
            dt += time.perf_counter() - t0
    return dt, len(frame_ids) * wl["pano_px"], n


def run_reference(args, dist):
    """The oracle as it stands, one bounded sample of the workload per step.

    A step is the oracle's full colour estimate of one frame plus its fused
    panorama on a strip of whole rows (computed pixel by pixel; the strip's
    output equals the same rows of its full-frame render), with the strip's
    time scaled to all rows. The strip height is set from the previous step's
    timing so that all steps together take about --ref-seconds seconds; frames
    cycle over at most four generated frames."""
    import numpy as np
    from oracle.pipeline import OracleStitcher
    if dist.rank != 0:
        return
    n_gen = max(1, min(args.frames, args.steps + args.warmup, 4))
    wl = make_workload(args.workload, n_gen, args.seed, "cpu", library=False)
    rig, seq = wl["rig"], wl["seq"]
    ex = rig.extra or {}
    o = OracleStitcher(rig.H, rig.cam_w, rig.cam_h, rig.pano_w, rig.pano_h, window=seq["window"],
                       max_flow=seq["max_flow"], projection=ex.get("projection", 0), cyl=ex.get("cyl"))
    host = [([f.numpy() for f in wl["frames"][t]], [f.numpy() for f in wl["fij"][t]],
             [f.numpy() for f in wl["fji"][t]]) for t in range(n_gen)]
    H, Wp = rig.pano_h, rig.pano_w
    per_step = args.ref_seconds / max(1, args.warmup + args.steps)
    rows = min(H, 32)
    times, strips, spent, cpu_s = [], [], 0.0, 0.0
    pool = one_thread()
    pool.__enter__()
    for s in range(args.warmup + args.steps):
        fr, a, b = host[s % n_gen]
        r0 = (s * 97) % (H - rows + 1)
        ys, xs = np.meshgrid(np.arange(r0, r0 + rows), np.arange(Wp), indexing="ij")
        c0 = time.process_time()
        t0 = time.perf_counter()
        o.estimate_color(fr)
        t1 = time.perf_counter()
        o.pixels(fr, a, b, xs.ravel(), ys.ravel())
        t2 = time.perf_counter()
        if s >= args.warmup:
            times.append((t1 - t0) + (t2 - t1) * H / rows)
            strips.append(rows)
            spent += t2 - t0
            cpu_s += time.process_time() - c0
        rows = int(min(H, max(8, (per_step - (t1 - t0)) / max((t2 - t1) / rows, 1e-9))))
    pool.__exit__(None, None, None)
    ms = 1e3 * sum(times) / len(times)
    value = wl["pano_px"] / (ms / 1e3) / 1e6
    sample = (f"per step: the full colour estimate of one frame plus the fused panorama on a strip of "
              f"{min(strips)}-{max(strips)} of its {H} rows (all {Wp} columns), strip time scaled to "
              f"{H} rows; {len(times)} timed steps over {n_gen} generated frames, {spent:.1f} s measured, "
              f"process CPU time / wall time {cpu_s / max(spent, 1e-9):.2f}")
    cpu = {"value": value, "unit": UNIT, "cores": max(1, round(cpu_s / max(spent, 1e-9))), "kind": "oracle",
           "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} rig -> {Wp}x{H} planar, FP64 CPU oracle, "
                                   "1 frame per step (bounded sample, scaled)",
                       "frames_per_step": 1},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)

# --------------------------------------------------------------------------- #
# batched / learned / cylindrical comparisons (outside the timed main step)
# --------------------------------------------------------------------------- #
def _time(fn, stream, steps, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _flat_seq(wls, F):
    fr, fij, fji = [], [], []
    for t in range(F):
        for w in wls:
            fr += w["frames"][t]
            fij += w["fij"][t]
            fji += w["fji"][t]
    return fr, fij, fji


def run_extras(args, dev, stream, ctxs):
    """The batched form (four rigs of uneven geometry, FP16 intermediates,
    one persistent fuse launch per frame) against the same rigs stitched one
    after the other; the learned estimator against the plain one; and the
    cylindrical 8 x 3840x2160 rig in its full form (learned estimate, FP16
    intermediates, batched launch) against its plain form."""
    import torch
    from paper_2308_09209_b300 import learned
    from paper_2308_09209_b300 import stitch as S
    from synth import BATCH_RIGS, make_window_pairs
    out = {}

    # batched vs plain
    F = 8
    wls = [make_workload(n, F, 20 + i, dev) for i, n in enumerate(BATCH_RIGS)]
    for w in wls:
        w["cfg"].flags = S.STITCH_FP16_INTERMEDIATE
    sts = [S.Stitcher(w["cfg"]) for w in wls]
    ctxs.extend(sts)
    b = S.stitch_batch_create([st.ctx for st in sts])
    panos = [torch.empty((3, w["cfg"].pano_h, w["cfg"].pitch), dtype=torch.uint8, device=dev)
             for _ in range(F) for w in wls]
    fr, fij, fji = _flat_seq(wls, F)
    shapes, ms_shapes = S.stitch_batch_autotune(b, fr[:sum(len(w["frames"][0]) for w in wls)],
                                               fij[:sum(len(w["fij"][0]) for w in wls)],
                                               fji[:sum(len(w["fji"][0]) for w in wls)], panos[:len(wls)], reps=3)
    alone = [S.Stitcher(w["cfg"]) for w in wls]
    ctxs.extend(alone)
    for st, sh in zip(alone, shapes):
        S.stitch_set_tile_shape(st.ctx, sh)
    per = []
    for w, st in zip(wls, alone):
        pp = [torch.empty((3, w["cfg"].pano_h, w["cfg"].pitch), dtype=torch.uint8, device=dev) for _ in range(F)]
        per.append(([f for t in range(F) for f in w["frames"][t]], [f for t in range(F) for f in w["fij"][t]],
                    [f for t in range(F) for f in w["fji"][t]], pp))

    def seq_all():
        for st, (a, c, d, pp) in zip(alone, per):
            S.stitch_sequence(st.ctx, F, a, c, d, pp, stream)

    def batch_all():
        S.stitch_batch_sequence(b, F, fr, fij, fji, panos, stream)

    # alternate the two forms, five repeats each, so that clock or neighbour
    # drift hits both alike; every repeat times 5 sequences of F frames
    reps_b, reps_p = [], []
    for _ in range(5):
        reps_b.append(_time(batch_all, stream, 5))
        reps_p.append(_time(seq_all, stream, 5))
    speedups = sorted(p / q for p, q in zip(reps_p, reps_b))
    ms_b, ms_p = sorted(reps_b)[2], sorted(reps_p)[2]
    px = F * sum(w["pano_px"] for w in wls)
    # frame 0 of every rig through a fresh batch, for the oracle check of the CPU-baseline leg
    fresh = [S.Stitcher(w["cfg"]) for w in wls]
    ctxs.extend(fresh)
    bf0 = S.stitch_batch_create([st.ctx for st in fresh])
    p0 = [torch.empty((3, w["cfg"].pano_h, w["cfg"].pitch), dtype=torch.uint8, device=dev) for w in wls]
    S.stitch_batch_sequence(bf0, 1, fr[:sum(len(w["frames"][0]) for w in wls)], fij[:sum(len(w["fij"][0]) for w in wls)],
                            fji[:sum(len(w["fji"][0]) for w in wls)], p0, stream)
    stream.synchronize()
    S.stitch_batch_destroy(bf0)
    out["_batched_check"] = [dict(rig=w["rig"], seq=w["seq"], flags=w["cfg"].flags,
                                  frames=[f.cpu().numpy() for f in w["frames"][0]],
                                  fij=[f.cpu().numpy() for f in w["fij"][0]],
                                  fji=[f.cpu().numpy() for f in w["fji"][0]], pano=p.cpu().numpy())
                             for w, p in zip(wls, p0)]
    out["batched"] = {"rigs": list(BATCH_RIGS), "frames_per_step": F, "intermediate": "fp16",
                      "tile_shapes": [S.TILE_SHAPES[sh] for sh in shapes],
                      "autotune_ms": [[round(float(m), 4) for m in row] for row in ms_shapes],
                      "batched_mpix_s": px / (ms_b / 1e3) / 1e6, "one_rig_at_a_time_mpix_s": px / (ms_p / 1e3) / 1e6,
                      "speedup": ms_p / ms_b, "speedup_per_repeat": speedups,
                      "speedup_min": speedups[0], "speedup_max": speedups[-1],
                      "repeats": "5 alternating repeats of each form (median reported); speedup_per_repeat "
                                 "pairs repeat k of one form with repeat k of the other"}
    S.stitch_batch_destroy(b)
    for st in sts + alone:
        st.close()
    del wls, panos, per, fr, fij, fji
    torch.cuda.empty_cache()

    # learned vs plain
    n_pairs, n_epochs = 200000, 40       # the learned configuration's 200k training pairs
    t0 = time.perf_counter()
    # each side three frames of the same crop of a moving scene: the window-pooled
    # overlap histograms the estimator sees on a rig (window 3)
    pairs, _ = make_window_pairs(n_pairs, seed=1, device=dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    feat, targ, _, flags = learned.label_pairs(pairs)
    t2 = time.perf_counter()
    net, hist = learned.train(feat, targ, epochs=n_epochs, batch=512, lr=1e-3, seed=1, mask=flags == 0)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    del pairs
    gain = learned.evaluate_gain(net, seeds=(201, 202), n_frames=8, objects=6)
    # training arithmetic: forward + two backward GEMMs per layer, 2 flops per multiply-add
    macs = 1536 * 512 + 512 * 512 + 512 * 256 + 256 * 16
    steps_pairs = (int((flags == 0).sum()) // 512) * 512 * n_epochs
    out["learned"] = {"train_pairs": n_pairs, "epochs": n_epochs, "final_loss": hist[-1],
                      "pairs": "two 128x96 crops of a synthetic scene under independent responses, each side "
                               "three frames of the moving scene stacked (window-pooled like a rig's overlap)",
                      "generate_s": t1 - t0, "label_s": t2 - t1, "train_s": t3 - t2,
                      "gemm_engine": "tcgen05", "train_tflops": 3 * 2 * macs * steps_pairs / (t3 - t2) / 1e12,
                      **gain}

    # cylindrical large rig: full form vs plain form on the same frames; a step
    # is the configuration's 120-frame sequence, cycling over 8 rendered frames
    # and 8 output panoramas (frame t + 8 is fused only after frame t, through
    # the colour-slot ring)
    F, n_r = 120, 8
    wl = make_workload("8x3840x2160cyl", n_r, 0, dev)
    fr = [f for t in range(F) for f in wl["frames"][t % n_r]]
    a = [f for t in range(F) for f in wl["fij"][t % n_r]]
    c = [f for t in range(F) for f in wl["fji"][t % n_r]]
    pr = [torch.empty((3, wl["cfg"].pano_h, wl["cfg"].pitch), dtype=torch.uint8, device=dev) for _ in range(n_r)]
    pp = [pr[t % n_r] for t in range(F)]
    plain = S.Stitcher(wl["cfg"])
    ctxs.append(plain)
    ms_plain = _time(lambda: S.stitch_sequence(plain.ctx, F, fr, a, c, pp, stream), stream, 3)
    S.stitch_window_fallbacks(plain.ctx, reset=True)
    S.stitch_sequence(plain.ctx, n_r, fr[:n_r * 8], a[:n_r * 7], c[:n_r * 7], pp[:n_r], stream)
    stream.synchronize()
    cyl_fb = S.stitch_window_fallbacks(plain.ctx, reset=True) / n_r
    wl["cfg"].flags = S.STITCH_FP16_INTERMEDIATE | S.STITCH_LEARNED
    full = S.Stitcher(wl["cfg"])
    ctxs.append(full)
    S.stitch_attach_mlp(full.ctx, net.h)
    bf = S.stitch_batch_create([full.ctx])
    shapes_full, _ = S.stitch_batch_autotune(bf, fr[:8], a[:7], c[:7], pp[:1], reps=2)
    ms_full = _time(lambda: S.stitch_batch_sequence(bf, F, fr, a, c, pp, stream), stream, 3)
    n_l, n_f = S.stitch_learned_stats(full.ctx)
    px = F * wl["pano_px"]
    rig = wl["rig"]
    out["cylindrical"] = {"workload": f"8x3840x2160 cylindrical rig -> {rig.pano_w}x{rig.pano_h}, window "
                                      f"{wl['seq']['window']}, max flow {wl['seq']['max_flow']} px, "
                                      f"{wl['seq']['objects']} moving objects, {F} frames per step "
                                      f"(cycling over {n_r} rendered frames)",
                          "plain_mpix_s": px / (ms_plain / 1e3) / 1e6,
                          "full_form_mpix_s": px / (ms_full / 1e3) / 1e6,
                          "full_form": "learned estimate with fallback, fp16 intermediates, batched launch, "
                                       f"tile {S.TILE_SHAPES[shapes_full[0]]}",
                          "learned_fallback_rate": n_f / max(n_l + n_f, 1),
                          "window_fallbacks_per_frame": cyl_fb,
                          "tile_shape_plain": list(S.stitch_tile_shape(plain.ctx)[1]),
                          "path_bytes_per_frame": wl["in_bytes"] + wl["flow_bytes"] + wl["out_bytes"]}
    S.stitch_batch_destroy(bf)
    net.close()
    return out


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
    # pick the fuse tile shape for this rig with the library's autotuner (one frame, outside the timed region)
    shape_ms = []
    if args.tile_shape < 0:
        S.stitch_estimate_color(st.ctx, wl["frames"][0], stream)
        shape, shape_ms = S.stitch_autotune(st.ctx, wl["frames"][0], wl["fij"][0], wl["fji"][0], panos[0], reps=5)
    st.close()
    ctxs.remove(st)
    st = S.Stitcher(cfg)                 # a fresh context with the tuned shape recorded for this rig
    ctxs.append(st)
    if args.tile_shape >= 0:
        S.stitch_set_tile_shape(st.ctx, args.tile_shape)
    torch.cuda.synchronize()

    def step():
        S.stitch_sequence(st.ctx, F, frames, fij, fji, panos, stream)

    # The autotuner times the fuse kernels alone; a shape it prefers over the
    # default is confirmed on the whole overlapped sequence (both shapes, a few
    # steps each, outside the timed region) and kept only if it is faster there.
    shape_check = None
    tuned = S.stitch_tile_shape(st.ctx)[0]
    if args.tile_shape < 0 and tuned != 0:
        ms_tuned = _time(step, stream, 3)
        S.stitch_set_tile_shape(st.ctx, 0)
        ms_default = _time(step, stream, 3)
        if ms_tuned < ms_default:
            S.stitch_set_tile_shape(st.ctx, tuned)
        shape_check = {"autotuner": list(S.TILE_SHAPES[tuned]),
                       "sequence_ms": {"x".join(map(str, S.TILE_SHAPES[tuned])): ms_tuned,
                                       "x".join(map(str, S.TILE_SHAPES[0])): ms_default}}

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
    # fuse tiles and pre-warp pieces whose source window did not fit in shared
    # memory (they take the per-pixel path with taps from global memory), per frame
    S.stitch_window_fallbacks(st.ctx, reset=True)
    step()
    stream.synchronize()
    win_fb = S.stitch_window_fallbacks(st.ctx, reset=True) / F

    # The same stages serialised: direct calls on one stream, one frame after
    # another, with the library's stage events around each launch group, so
    # that every stage time is the duration of its own kernels alone.
    sts = S.Stitcher(cfg)
    ctxs.append(sts)
    if args.tile_shape >= 0:
        S.stitch_set_tile_shape(sts.ctx, args.tile_shape)
    pano_s = torch.empty((3, cfg.pano_h, cfg.pitch), dtype=torch.uint8, device=dev)
    for t in range(min(F, 4)):
        S.stitch_estimate_color(sts.ctx, wl["frames"][t], stream)
        S.stitch_frame(sts.ctx, wl["frames"][t], wl["fij"][t], wl["fji"][t], pano_s, stream)
    stream.synchronize()
    S.stitch_profile(sts.ctx, True)
    S.stitch_profile_read(sts.ctx)
    for t in range(F):
        S.stitch_estimate_color(sts.ctx, wl["frames"][t], stream)
        S.stitch_frame(sts.ctx, wl["frames"][t], wl["fij"][t], wl["fji"][t], pano_s, stream)
    stream.synchronize()
    rs = S.stitch_profile_read(sts.ctx)
    S.stitch_profile(sts.ctx, False)
    serial = {k[:-3]: rs[k] / max(rs[k[:-3] + "_n"], 1) for k in ("stats_ms", "estimate_ms", "prewarp_ms", "fuse_ms")}
    sts.close()
    ctxs.remove(sts)
    del pano_s

    fuse_ms = acc["fuse_ms"] / max(acc["fuse_n"], 1)
    prewarp_ms = acc["prewarp_ms"] / max(acc["prewarp_n"], 1)
    stats_ms = acc["stats_ms"] / max(acc["stats_n"], 1)
    est_ms = acc["estimate_ms"] / max(acc["estimate_n"], 1)
    # the fused warp stage of one frame, its kernels running alone
    warp_ms = serial["fuse"] + serial["prewarp"]
    fuse_bytes = wl["in_bytes"] + wl["flow_bytes"] + wl["out_bytes"]
    peak, peak_kind = measured_peaks()
    achieved = fuse_bytes / (warp_ms / 1e3) / 1e9
    traffic = traffic_from_profile(args.workload)
    issue_prof = issue_from_profiles(args.workload)
    issue_instr = issue_prof[0] if issue_prof else None
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
    link = host_link_gbs(dev, stream)
    # the copies bound e2e: per frame, the larger of copy-in and copy-out time
    frame_copy_s = max(h2d / n_e2e / (link["h2d_gbs"] * 1e9), d2h / n_e2e / (link["d2h_gbs"] * 1e9))
    link["e2e_bound_mpix_s"] = dist.world * wl["pano_px"] / frame_copy_s / 1e6
    link["e2e_frac_of_bound"] = e2e_value / link["e2e_bound_mpix_s"]

    extras = {}
    if dist.rank == 0 and dist.world == 1 and not args.no_extras:
        # the same workload with FP16 band intermediates (coordinates and arithmetic stay FP32)
        cfg16 = S.Config(cfg.cam_w, cfg.cam_h, cfg.H, cfg.pano_w, cfg.pano_h, window=cfg.window,
                         max_flow=cfg.max_flow, flags=S.STITCH_FP16_INTERMEDIATE)
        st16 = S.Stitcher(cfg16)
        ctxs.append(st16)
        ms16 = _time(lambda: S.stitch_sequence(st16.ctx, F, frames, fij, fji, panos, stream), stream,
                     max(3, min(args.steps, 20)), 2)
        extras["fp16_intermediates"] = {"value": F * wl["pano_px"] / (ms16 / 1e3) / 1e6, "unit": UNIT,
                                        "ms_per_step": ms16}
        del panos, h_frames, h_fij, h_fji, h_out
        extras.update(run_extras(args, dev, stream, ctxs))
        # homography refinement from frame 0's band flows (synchronous call; host clock)
        n_cams = len(wl["rig"].cam_w)
        S.stitch_refine_homographies(st.ctx, wl["fij"][0], wl["fji"][0], n_cams)
        t0 = time.perf_counter()
        for _ in range(10):
            S.stitch_refine_homographies(st.ctx, wl["fij"][0], wl["fji"][0], n_cams)
        refine_ms = (time.perf_counter() - t0) / 10 * 1e3
        band_px = int(sum(int(f.shape[0]) * int(f.shape[1]) for f in wl["fij"][0]))
        extras["refine_homographies"] = {"ms_per_call": refine_ms, "pairs": n_cams - 1,
                                         "band_px": band_px,
                                         "what": "8 exact medians per pair (radix selection, 4 passes), "
                                                 "then the composed float64 homographies"}
        # band optical flow of frame 0 (stream-ordered; CUDA events on the stream)
        fl_ij = [torch.empty_like(f) for f in wl["fij"][0]]
        fl_ji = [torch.empty_like(f) for f in wl["fji"][0]]
        ms_flow = _time(lambda: S.stitch_estimate_flow(st.ctx, wl["frames"][0], fl_ij, fl_ji, stream), stream, 10, 2)
        # the whole per-frame method with the library's own flow: flow, colour estimate, stitch
        stf = S.Stitcher(cfg)
        ctxs.append(stf)
        pano1 = torch.empty((3, cfg.pano_h, cfg.pitch), dtype=torch.uint8, device=dev)
        nf = min(F, 8)

        def with_flow():
            for t in range(nf):
                S.stitch_estimate_flow(stf.ctx, wl["frames"][t], fl_ij, fl_ji, stream)
                S.stitch_estimate_color(stf.ctx, wl["frames"][t], stream)
                S.stitch_frame(stf.ctx, wl["frames"][t], fl_ij, fl_ji, pano1, stream)

        ms_wf = _time(with_flow, stream, 3, 1) / nf
        extras["estimate_flow"] = {"ms_per_frame": ms_flow, "pairs": n_cams - 1, "band_px": band_px,
                                   "what": "float32 band pre-warp of both cameras, integer luminance, 3-level "
                                           "7x7 block matching both ways, sub-pixel parabola",
                                   "with_stitch_mpix_s": wl["pano_px"] / (ms_wf / 1e3) / 1e6,
                                   "with_stitch": "per frame: stitch_estimate_flow, stitch_estimate_color, "
                                                  "stitch_frame with those flows (direct calls, one stream)"}
        # the temporal-window study (W = 1 vs 3 / 5 / 7), outside every timed region
        from paper_2308_09209_b300.study import window_study
        extras["window_study"] = window_study()

    cpu_baseline = None
    err = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        dt, px, outs, cpu_s = oracle_frames(wl, [0, 1], keep=True)
        single = {"value": px / dt / 1e6, "unit": UNIT, "cores": max(1, round(cpu_s / dt)),
                  "sample": f"frames 0-1 of the workload: estimate + full {wl['rig'].pano_w}x"
                            f"{wl['rig'].pano_h} panorama each, numpy float64, one thread (process CPU time / "
                            f"wall time {cpu_s / dt:.2f})"}
        hi = host_info()
        dta, pxa, na = oracle_all_cores(wl, [0, 1])
        # the other workloads of the CPU-baseline plan: the whole small rig, and one
        # frame of the 8 x 4K cylinder (its inputs rendered on the GPU, then copied)
        wl1 = make_workload("2x640x360", 8, args.seed, "cpu", library=False)
        d1, p1, _, c1 = oracle_frames(wl1, list(range(8)))
        d1a, p1a, _ = oracle_all_cores(wl1, list(range(8)))
        wl5 = make_workload("8x3840x2160cyl", 1, args.seed, dev, library=False)
        d5a, p5a, _ = oracle_all_cores(wl5, [0])
        del wl5
        cpu_baseline = {"value": pxa / dta / 1e6, "unit": UNIT, "cores": na, "kind": "oracle",
                        "sample": f"frames 0-1 of the workload: the colour estimate (serial) and the full "
                                  f"{wl['rig'].pano_w}x{wl['rig'].pano_h} panorama in strips of rows over {na} "
                                  f"spawned worker processes, numpy float64",
                        "host": hi, "single_thread": single,
                        "2x640x360_all_8_frames": {"single_thread_mpix_s": p1 / d1 / 1e6,
                                                   "all_cores_mpix_s": p1a / d1a / 1e6,
                                                   "single_thread_fps": 8 / d1, "all_cores_fps": 8 / d1a},
                        "8x3840x2160cyl_frame0": {"all_cores_mpix_s": p5a / d5a / 1e6, "all_cores_fps": 1 / d5a}}
        # the same two frames from a fresh context, compared with the oracle's panoramas
        st3 = S.Stitcher(cfg)
        ctxs.append(st3)
        g = []
        for t in (0, 1):
            st3.estimate_color(wl["frames"][t])
            g.append(st3.frame(wl["frames"][t], wl["fij"][t], wl["fji"][t]))
        torch.cuda.synchronize()
        err = oracle_error(g, outs, cfg.pano_w)
        # the same frames with FP16 band intermediates, against the oracle in that mode
        cfg16 = S.Config(cfg.cam_w, cfg.cam_h, cfg.H, cfg.pano_w, cfg.pano_h, window=cfg.window,
                         max_flow=cfg.max_flow, flags=S.STITCH_FP16_INTERMEDIATE)
        st4 = S.Stitcher(cfg16)
        ctxs.append(st4)
        g16 = []
        for t in (0, 1):
            st4.estimate_color(wl["frames"][t])
            g16.append(st4.frame(wl["frames"][t], wl["fij"][t], wl["fji"][t]))
        torch.cuda.synchronize()
        _, _, outs16, _ = oracle_frames(wl, [0, 1], keep=True, flags=S.STITCH_FP16_INTERMEDIATE)
        err = {"fp32_intermediates": err, "fp16_intermediates": oracle_error(g16, outs16, cfg.pano_w)}
        if "_batched_check" in extras:
            err["batched_rigs_frame0"] = oracle_check_rigs(extras["_batched_check"])


    # stats, estimate, band pre-warp, fuse (general pieces), fuse (band pieces), fuse (fully covered own pieces)
    launches = args.steps * F * 6
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
                       "stage_ms_per_frame": {"stats": serial["stats"], "estimate": serial["estimate"],
                                              "band_prewarp": serial["prewarp"], "fuse": serial["fuse"]},
                       "stage_timing": "serialised: direct calls on one stream, CUDA events around each "
                                       "stage's launches (the roofline's kernel time)",
                       "stage_ms_in_graph": {"stats": stats_ms, "estimate": est_ms, "band_prewarp": prewarp_ms,
                                             "fuse": fuse_ms},
                       "stage_in_graph_timing": stage_timing + " (stages overlap across frames and streams)",
                       "status": rc, "parallelism": f"replicas x{dist.world}",
                       "tile_shape": list(S.stitch_tile_shape(st.ctx)[1]),
                       "autotune_ms": [round(float(m), 4) for m in shape_ms],
                       "tile_shape_check": shape_check,
                       "window_fallbacks_per_frame": win_fb,
                       "oracle_error": err, **extras},
            "roofline": {"bound": "hbm", "kernel": "fused warp stage of a frame (k_prewarp_band + k_fuse + k_fuse_band + k_fuse_own)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": fuse_bytes},
            "cpu_baseline": cpu_baseline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "frames_per_step": n_e2e, "host_link": link},
            "clocks": clk,
            "gpu_launches": launches,
        }
        line["config"].pop("_batched_check", None)
        if issue_instr and clk and clk.get("sm_mhz"):
            # The path is bound by instruction issue rather than HBM: warp
            # instructions of all five kernels per frame (ncu, one capture of
            # this workload) over the live frame time, against 148 SMs x 4
            # schedulers x one warp instruction per clock at the sampled clock.
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak_issue = sms * 4 * clk["sm_mhz"] * 1e6
            achieved_issue = issue_instr / (ms / F / 1e3)
            line["config"]["issue"] = {"warp_instructions_per_frame": issue_instr,
                                       "achieved_warp_inst_per_s": achieved_issue,
                                       "peak_warp_inst_per_s": peak_issue, "frac": achieved_issue / peak_issue,
                                       "source": "ncu smsp__inst_executed.sum per kernel from profiles/"
                                                 f"{{fuse,stats,estimate}}_{args.workload}.md",
                                       "captured_tile_shape": list(issue_prof[1]),
                                       "bench_tile_shape": list(S.stitch_tile_shape(st.ctx)[1])}
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
