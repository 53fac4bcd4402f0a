"""Build the stitching library (libstitch.so) in-tree with nvcc for sm_103a.

Usage: python -m paper_2308_09209_b300.build [--force] [--verbose]
The shared library lands next to this file, where the Python binding loads it.
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libstitch.so")
SOURCES = ["host.cu", "k_stats.cu", "k_estimate.cu", "k_fuse.cu", "noalloc.cu", "k_pairs.cu", "k_mlp.cu", "k_learned.cu", "k_mlp_tc.cu",
           "k_refine.cu", "k_flow.cu", "k_corr.cu",
           "mlp_host.cu"]
HEADERS = ["stitch_internal.h", "estimate_common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "stitch.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, obj: str, verbose: bool):
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return subprocess.run(cmd, capture_output=True, text=True), cmd


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object in parallel, then link libstitch.so."""
    if not force and not _stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, f.replace(".cu", ".o")) for f in SOURCES]
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda a: _compile(*a, verbose),
                              [(os.path.join(CSRC, f), o) for f, o in zip(SOURCES, objs)]))
    for res, cmd in results:
        if verbose:
            print(" ".join(cmd))
            sys.stderr.write(res.stderr)
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("nvcc failed building libstitch.so")
    link = [_nvcc(), *ARCH, "--shared", "-o", LIB + ".tmp"] + objs
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed linking libstitch.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build(a.force, a.verbose))
