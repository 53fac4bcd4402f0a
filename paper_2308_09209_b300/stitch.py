"""Python binding of the C-ABI stitching library (include/stitch.h).

Argument marshalling only: every step of the stitching path runs in the CUDA
kernels of libstitch.so. Functions carry the same names as the C entry
points. Device buffers are torch CUDA tensors (their data pointers are passed
through); streams are torch.cuda.Stream objects or None (legacy default).
There is no CPU fallback: if libstitch.so is missing, using any entry point
raises.
"""
from __future__ import annotations

import ctypes
import os
import sys
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstitch.so")

STITCH_OK = 0
STITCH_EINVAL = -1
STITCH_ENOMEM = -2
STITCH_ECUDA = -3
STITCH_ESINGULAR = -4
STITCH_ETIMEOUT = -5
STITCH_EFALLBACK = 1

STITCH_BALANCE_OFF = 1
STITCH_FP16_INTERMEDIATE = 2
STITCH_FLOW_WEIGHTS_PRINTED = 4
STITCH_LEARNED = 8
STITCH_BALANCE_OUTPUT = 16
STITCH_PROJ_PLANAR = 0
STITCH_PROJ_CYLINDRICAL = 1

STITCH_MAX_CAMS = 8
STITCH_CURVE_FLOATS = 10
CURVE_FIELDS = ("m1", "m2", "d1", "d2", "s", "g1", "g2", "inv_m1", "inv_bm", "identity")


class StitchError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"stitch error {code}: {msg}")
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [
        ("n_cams", ctypes.c_int),
        ("cam_w", ctypes.POINTER(ctypes.c_int)),
        ("cam_h", ctypes.POINTER(ctypes.c_int)),
        ("cam_pitch", ctypes.POINTER(ctypes.c_int)),
        ("H", ctypes.POINTER(ctypes.c_double)),
        ("pano_w", ctypes.c_int),
        ("pano_h", ctypes.c_int),
        ("pano_pitch", ctypes.c_int),
        ("projection", ctypes.c_int),
        ("ref_cam", ctypes.c_int),
        ("window", ctypes.c_int),
        ("lambda_", ctypes.c_double),
        ("max_flow", ctypes.c_float),
        ("flags", ctypes.c_int),
        ("cyl_focal", ctypes.c_double),
        ("cyl_cx", ctypes.c_double),
        ("cyl_cy", ctypes.c_double),
    ]


_lib = None


def lib():
    """The loaded libstitch.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2308_09209_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, cfgp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_Config)
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "stitch_geometry": (ip, [cfgp, vp, vp]),
            "stitch_init": (ip, [cfgp, ctypes.POINTER(vp)]),
            "stitch_estimate_color": (ip, [vp, pp, vp]),
            "stitch_frame": (ip, [vp, pp, pp, pp, vp, vp]),
            "stitch_sequence": (ip, [vp, ip, pp, pp, pp, pp, vp]),
            "stitch_sequence_host": (ip, [vp, ip, pp, pp, pp, pp, vp]),
            "stitch_sync": (ip, [vp, vp]),
            "stitch_get_color": (ip, [vp, vp, vp, vp]),
            "stitch_get_pair_M": (ip, [vp, vp]),
            "stitch_get_frame_stats": (ip, [vp, vp, vp, vp, vp, vp, vp]),
            "stitch_get_bands": (ip, [vp, vp, vp]),
            "stitch_save_state": (ip, [vp, vp, ctypes.POINTER(ctypes.c_size_t)]),
            "stitch_load_state": (ip, [vp, vp, ctypes.c_size_t]),
            "stitch_profile": (ip, [vp, ip]),
            "stitch_profile_read": (ip, [vp, vp, vp]),
            "stitch_estimate_color_noalloc": (ip, [cfgp, pp, vp, vp, vp, vp]),
            "stitch_mlp_n_params": (ip, []),
            "stitch_mlp_create": (ip, [ip, ctypes.c_ulonglong, ctypes.POINTER(vp)]),
            "stitch_mlp_destroy": (None, [vp]),
            "stitch_mlp_set_gemm": (ip, [vp, ip]),
            "stitch_mlp_status": (ip, [vp]),
            "stitch_mlp_inject_error": (ip, [vp, ip]),
            "stitch_mlp_set_norm": (ip, [vp, vp, vp]),
            "stitch_mlp_get_params": (ip, [vp, vp]),
            "stitch_mlp_set_params": (ip, [vp, vp]),
            "stitch_mlp_forward": (ip, [vp, vp, ip, vp, vp]),
            "stitch_mlp_train_step": (ip, [vp, vp, vp, ip, ctypes.c_float, vp, vp]),
            "stitch_mlp_gradients": (ip, [vp, vp, vp, ip, vp, vp]),
            "stitch_pairs_label": (ip, [vp, ip, ip, ip, ctypes.c_double, vp, vp, vp, vp, vp]),
            "stitch_attach_mlp": (ip, [vp, vp]),
            "stitch_learned_stats": (ip, [vp, vp, vp]),
            "stitch_get_learned": (ip, [vp, vp, vp, vp]),
            "stitch_autotune": (ip, [vp, pp, pp, pp, vp, ip, vp, vp]),
            "stitch_tile_shape": (ip, [vp, vp, vp]),
            "stitch_set_tile_shape": (ip, [vp, ip]),
            "stitch_batch_create": (ip, [pp, ip, ctypes.POINTER(vp)]),
            "stitch_batch_sequence": (ip, [vp, ip, pp, pp, pp, pp, vp]),
            "stitch_batch_autotune": (ip, [vp, pp, pp, pp, pp, ip, vp, vp]),
            "stitch_batch_tile_shapes": (ip, [vp, vp]),
            "stitch_refine_homographies": (ip, [vp, pp, pp, vp, vp]),
            "stitch_estimate_flow": (ip, [vp, pp, pp, pp, vp]),
            "stitch_get_flow_luma": (ip, [vp, ip, ip, ip, vp, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
            "stitch_pair_M_correspondence": (ip, [vp, pp, vp]),
            "stitch_selftest_wait": (ip, [ip, ip]),
            "stitch_batch_destroy": (None, [vp]),
            "stitch_batch_last_error": (ctypes.c_char_p, [vp]),
            "stitch_n_pairs": (ip, [vp]),
            "stitch_window_fallbacks": (ip, [vp, ctypes.POINTER(ctypes.c_ulonglong), ip]),
            "stitch_get_output_hist": (ip, [vp, vp]),
            "stitch_last_error": (ctypes.c_char_p, [vp]),
            "stitch_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


@dataclass
class Config:
    """Python mirror of stitch_config (include/stitch.h)."""
    cam_w: Sequence[int]
    cam_h: Sequence[int]
    H: np.ndarray                       # (n_cams, 3, 3) camera -> panorama
    pano_w: int
    pano_h: int
    pano_pitch: Optional[int] = None    # default: pano_w rounded up to 16
    cam_pitch: Optional[Sequence[int]] = None
    ref_cam: int = -1
    window: int = 3
    lam: float = 0.05
    max_flow: float = 8.0
    flags: int = 0
    projection: int = 0                 # 0 planar, 1 cylindrical (H = camera pixel -> ray)
    cyl: Optional[Sequence[float]] = None   # (focal px/rad, cx, cy) for the cylindrical projection
    _keep: list = field(default_factory=list, repr=False)

    @property
    def n_cams(self) -> int:
        return len(self.cam_w)

    @property
    def pitch(self) -> int:
        return self.pano_pitch if self.pano_pitch is not None else (self.pano_w + 15) // 16 * 16

    def c_struct(self) -> _Config:
        n = self.n_cams
        w = (ctypes.c_int * n)(*[int(v) for v in self.cam_w])
        h = (ctypes.c_int * n)(*[int(v) for v in self.cam_h])
        Hs = np.ascontiguousarray(np.asarray(self.H, dtype=np.float64).reshape(n, 9))
        Hc = (ctypes.c_double * (9 * n))(*Hs.ravel().tolist())
        pc = None
        if self.cam_pitch is not None:
            pc = (ctypes.c_int * n)(*[int(v) for v in self.cam_pitch])
        self._keep[:] = [w, h, Hc, pc]
        c = _Config()
        c.n_cams = n
        c.cam_w = w
        c.cam_h = h
        c.cam_pitch = pc if pc is not None else ctypes.POINTER(ctypes.c_int)()
        c.H = Hc
        c.pano_w = int(self.pano_w)
        c.pano_h = int(self.pano_h)
        c.pano_pitch = int(self.pitch)
        c.projection = int(self.projection)
        if self.cyl is not None:
            c.cyl_focal, c.cyl_cx, c.cyl_cy = (float(v) for v in self.cyl)
        c.ref_cam = int(self.ref_cam)
        c.window = int(self.window)
        c.lambda_ = float(self.lam)
        c.max_flow = float(self.max_flow)
        c.flags = int(self.flags)
        return c


def _check(rc: int, ctx=None, allow=(STITCH_OK,)):
    if rc in allow:
        return rc
    msg = lib().stitch_last_error(ctx)
    raise StitchError(rc, msg.decode() if msg else "")


def _ptrs(tensors) -> ctypes.Array:
    vals = []
    for t in tensors:
        vals.append(ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr()))
    return (ctypes.c_void_p * max(1, len(vals)))(*vals)


def _host_ptrs(arrays) -> ctypes.Array:
    vals = []
    for a in arrays:
        if hasattr(a, "data_ptr"):
            vals.append(ctypes.c_void_p(a.data_ptr()))
        else:
            vals.append(ctypes.c_void_p(a.ctypes.data))
    return (ctypes.c_void_p * max(1, len(vals)))(*vals)


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def stitch_geometry(cfg: Config):
    """Host-only geometry: (bands (n_pairs, 4), rects (n_pairs, 2, 4)) int32."""
    c = cfg.c_struct()
    npairs = max(cfg.n_cams - 1, 1)
    bands = np.zeros((npairs, 4), dtype=np.int32)
    rects = np.zeros((npairs, 2, 4), dtype=np.int32)
    rc = lib().stitch_geometry(ctypes.byref(c), bands.ctypes.data, rects.ctypes.data)
    _check(rc)
    return bands, rects


def stitch_init(cfg: Config):
    c = cfg.c_struct()
    out = ctypes.c_void_p()
    _check(lib().stitch_init(ctypes.byref(c), ctypes.byref(out)))
    return out


def stitch_estimate_color(ctx, frames, stream=None) -> int:
    return _check(lib().stitch_estimate_color(ctx, _ptrs(frames), _stream(stream)), ctx)


def stitch_frame(ctx, frames, flows_ij, flows_ji, pano, stream=None) -> int:
    return _check(lib().stitch_frame(ctx, _ptrs(frames), _ptrs(flows_ij), _ptrs(flows_ji),
                                     ctypes.c_void_p(pano.data_ptr()), _stream(stream)), ctx)


def stitch_sequence(ctx, n_frames, frames, flows_ij, flows_ji, panos, stream=None) -> int:
    """frames: flat frame-major list (n_frames * n_cams); flows: n_frames * n_pairs; panos: n_frames."""
    return _check(lib().stitch_sequence(ctx, int(n_frames), _ptrs(frames), _ptrs(flows_ij), _ptrs(flows_ji),
                                        _ptrs(panos), _stream(stream)), ctx)


def stitch_sequence_host(ctx, n_frames, frames, flows_ij, flows_ji, panos, stream=None) -> int:
    """As stitch_sequence with host arrays (numpy or pinned torch CPU tensors)."""
    return _check(lib().stitch_sequence_host(ctx, int(n_frames), _host_ptrs(frames), _host_ptrs(flows_ij),
                                             _host_ptrs(flows_ji), _host_ptrs(panos), _stream(stream)),
                  ctx, allow=(STITCH_OK, STITCH_ESINGULAR))


def stitch_sync(ctx, stream=None) -> int:
    return _check(lib().stitch_sync(ctx, _stream(stream)), ctx, allow=(STITCH_OK, STITCH_ESINGULAR))


def stitch_get_color(ctx, n_cams: int):
    """(status, M (n_cams, 3, 3) float64, curve dict of (3,) arrays, frame index)."""
    M = np.zeros((n_cams, 9), dtype=np.float64)
    curve = np.zeros((3, STITCH_CURVE_FLOATS), dtype=np.float32)
    T = ctypes.c_int(0)
    rc = _check(lib().stitch_get_color(ctx, M.ctypes.data, curve.ctypes.data, ctypes.byref(T)), ctx,
                allow=(STITCH_OK, STITCH_ESINGULAR))
    cd = {name: curve[:, i].copy() for i, name in enumerate(CURVE_FIELDS)}
    return rc, M.reshape(n_cams, 3, 3), cd, T.value


def stitch_get_pair_M(ctx, n_pairs: int) -> np.ndarray:
    M = np.zeros((n_pairs, 9), dtype=np.float64)
    _check(lib().stitch_get_pair_M(ctx, M.ctypes.data), ctx)
    return M.reshape(n_pairs, 3, 3)


def stitch_get_frame_stats(ctx, n_pairs: int) -> dict:
    pooled = np.zeros((3, 256), dtype=np.uint32)
    Hi = np.zeros((n_pairs, 3, 256), dtype=np.uint32)
    Hj = np.zeros((n_pairs, 3, 256), dtype=np.uint32)
    Wv = np.zeros((n_pairs, 6, 256), dtype=np.uint32)
    A = np.zeros((n_pairs, 9), dtype=np.uint64)
    B = np.zeros((n_pairs, 9), dtype=np.uint64)
    _check(lib().stitch_get_frame_stats(ctx, pooled.ctypes.data, Hi.ctypes.data, Hj.ctypes.data, Wv.ctypes.data,
                                        A.ctypes.data, B.ctypes.data), ctx)
    return dict(pooled=pooled, Hi=Hi, Hj=Hj, Wv=Wv, A=A.reshape(n_pairs, 3, 3), B=B.reshape(n_pairs, 3, 3))


def stitch_get_bands(ctx, n_pairs: int):
    bands = np.zeros((n_pairs, 4), dtype=np.int32)
    rects = np.zeros((n_pairs, 2, 4), dtype=np.int32)
    _check(lib().stitch_get_bands(ctx, bands.ctypes.data, rects.ctypes.data), ctx)
    return bands, rects


def stitch_save_state(ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().stitch_save_state(ctx, None, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().stitch_save_state(ctx, buf, ctypes.byref(n)), ctx)
    return buf.raw[: n.value]


def stitch_load_state(ctx, blob: bytes) -> int:
    buf = ctypes.create_string_buffer(blob, len(blob))
    return _check(lib().stitch_load_state(ctx, buf, len(blob)), ctx)


def stitch_profile(ctx, enable: bool) -> int:
    return _check(lib().stitch_profile(ctx, 1 if enable else 0), ctx)


def stitch_profile_read(ctx) -> dict:
    """Per-stage GPU milliseconds and launch counts since the last read."""
    ms = np.zeros(4, dtype=np.float64)
    cnt = np.zeros(4, dtype=np.int32)
    _check(lib().stitch_profile_read(ctx, ms.ctypes.data, cnt.ctypes.data), ctx)
    return dict(stats_ms=float(ms[0]), estimate_ms=float(ms[1]), fuse_ms=float(ms[2]), prewarp_ms=float(ms[3]),
                stats_n=int(cnt[0]), estimate_n=int(cnt[1]), fuse_n=int(cnt[2]), prewarp_n=int(cnt[3]))


def stitch_estimate_color_noalloc(cfg: Config, frames, M_out, curve_out, flags_out=None, stream=None) -> int:
    """Single-frame colour estimate into caller-owned device tensors, with no
    device allocation inside the library (for callers that cannot allocate).
    M_out: float64 CUDA tensor of n_cams * 9; curve_out: float32 CUDA tensor of
    3 * STITCH_CURVE_FLOATS; flags_out: optional int32 CUDA tensor of 1."""
    import torch

    def _need(t, name, dtype, n):
        if (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous()
                or t.numel() < n):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of at least {n} elements")

    _need(M_out, "M_out", torch.float64, cfg.n_cams * 9)
    _need(curve_out, "curve_out", torch.float32, 3 * STITCH_CURVE_FLOATS)
    if flags_out is not None:
        _need(flags_out, "flags_out", torch.int32, 1)
    c = cfg.c_struct()
    fl = ctypes.c_void_p(flags_out.data_ptr()) if flags_out is not None else None
    return _check(lib().stitch_estimate_color_noalloc(ctypes.byref(c), _ptrs(frames),
                                                      ctypes.c_void_p(M_out.data_ptr()),
                                                      ctypes.c_void_p(curve_out.data_ptr()), fl,
                                                      _stream(stream)))


# --------------------------------------------------------------------------- #
# Learned estimator
# --------------------------------------------------------------------------- #
STITCH_MLP_IN = 1536
STITCH_MLP_OUT = 12


def _dp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def stitch_mlp_n_params() -> int:
    return lib().stitch_mlp_n_params()


def stitch_mlp_create(max_batch: int, seed: int):
    out = ctypes.c_void_p()
    _check(lib().stitch_mlp_create(max_batch, seed, ctypes.byref(out)))
    return out


def stitch_mlp_destroy(mlp) -> None:
    if mlp is not None and mlp.value:
        lib().stitch_mlp_destroy(mlp)


STITCH_MLP_GEMM_MMA_SYNC = 0
STITCH_MLP_GEMM_TCGEN05 = 1


def stitch_mlp_set_gemm(mlp, engine: int) -> int:
    return _check(lib().stitch_mlp_set_gemm(mlp, engine))


def stitch_mlp_status(mlp) -> int:
    return _check(lib().stitch_mlp_status(mlp))


def stitch_mlp_inject_error(mlp, word: int) -> int:
    """Write a timed-out kernel's error word (tests of the status handling)."""
    return _check(lib().stitch_mlp_inject_error(mlp, word))


def stitch_mlp_set_norm(mlp, mu, sd) -> int:
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    sd = np.ascontiguousarray(sd, dtype=np.float32)
    assert mu.size == STITCH_MLP_OUT and sd.size == STITCH_MLP_OUT
    return _check(lib().stitch_mlp_set_norm(mlp, mu.ctypes.data, sd.ctypes.data))


def stitch_mlp_get_params(mlp) -> np.ndarray:
    out = np.zeros(stitch_mlp_n_params(), dtype=np.float32)
    _check(lib().stitch_mlp_get_params(mlp, out.ctypes.data))
    return out


def stitch_mlp_set_params(mlp, params) -> int:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == stitch_mlp_n_params()
    return _check(lib().stitch_mlp_set_params(mlp, p.ctypes.data))


def stitch_mlp_forward(mlp, x, batch: int, y, stream=None) -> int:
    """x: bfloat16 (or int16 bit patterns) CUDA tensor [batch, 1536]; y: float32 CUDA tensor [batch, 12]."""
    return _check(lib().stitch_mlp_forward(mlp, _dp(x), batch, _dp(y), _stream(stream)))


def stitch_mlp_train_step(mlp, x, t, batch: int, lr: float, loss=None, stream=None) -> int:
    return _check(lib().stitch_mlp_train_step(mlp, _dp(x), _dp(t), batch, lr, _dp(loss), _stream(stream)))


def stitch_mlp_gradients(mlp, x, t, batch: int):
    """(gradients float32 [n_params], loss) of one batch, without an update."""
    g = np.zeros(stitch_mlp_n_params(), dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(lib().stitch_mlp_gradients(mlp, _dp(x), _dp(t), batch, g.ctypes.data, loss.ctypes.data))
    return g, float(loss[0])


def stitch_pairs_label(pairs, n_pairs: int, patch_w: int, patch_h: int, lam: float, features, targets,
                       M=None, flags=None, stream=None) -> int:
    """Plain one-frame fit, features and targets of n_pairs independent pairs
    (uint8 CUDA tensor [n_pairs, 2, patch_h, patch_w, 3])."""
    return _check(lib().stitch_pairs_label(_dp(pairs), n_pairs, patch_w, patch_h, lam, _dp(features), _dp(targets),
                                           _dp(M), _dp(flags), _stream(stream)))


def stitch_attach_mlp(ctx, mlp) -> int:
    return _check(lib().stitch_attach_mlp(ctx, mlp), ctx)


def stitch_learned_stats(ctx):
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().stitch_learned_stats(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def stitch_get_learned(ctx, n_pairs: int):
    """(M_hat [n_pairs, 3, 3], residual [n_pairs], used [n_pairs]) of the latest frame."""
    M = np.zeros((max(n_pairs, 1), 3, 3), dtype=np.float64)
    r = np.zeros(max(n_pairs, 1), dtype=np.float64)
    u = np.zeros(max(n_pairs, 1), dtype=np.int32)
    _check(lib().stitch_get_learned(ctx, M.ctypes.data, r.ctypes.data, u.ctypes.data), ctx)
    return M[:n_pairs], r[:n_pairs], u[:n_pairs]


class Mlp:
    """Owner of a network handle (stitch_mlp)."""

    def __init__(self, max_batch: int = 256, seed: int = 0):
        self.max_batch = max_batch
        self.h = stitch_mlp_create(max_batch, seed)

    def close(self):
        if self.h is not None:
            stitch_mlp_destroy(self.h)
        self.h = None

    def __del__(self):
        if sys is None or sys.is_finalizing():
            return
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- #
# Tile shapes, autotuner, batched rigs
# --------------------------------------------------------------------------- #
STITCH_TILE_SHAPES = 6
STITCH_BATCH_MAX_RIGS = 16
TILE_SHAPES = ((64, 32), (64, 16), (32, 32), (128, 16), (32, 16), (128, 32))


def stitch_autotune(ctx, frames, flows_ij, flows_ji, pano, reps: int = 5):
    """(chosen shape index, mean ms per fuse launch for every shape, -1 = does not fit)."""
    ms = np.zeros(STITCH_TILE_SHAPES, dtype=np.float32)
    shape = ctypes.c_int(0)
    _check(lib().stitch_autotune(ctx, _ptrs(frames), _ptrs(flows_ij), _ptrs(flows_ji), ctypes.c_void_p(pano.data_ptr()),
                                 reps, ctypes.byref(shape), ms.ctypes.data), ctx)
    return shape.value, ms


def stitch_tile_shape(ctx):
    w, h = ctypes.c_int(), ctypes.c_int()
    idx = lib().stitch_tile_shape(ctx, ctypes.byref(w), ctypes.byref(h))
    return idx, (w.value, h.value)


def stitch_set_tile_shape(ctx, shape: int) -> int:
    return _check(lib().stitch_set_tile_shape(ctx, shape), ctx)


def _batch_check(rc, b):
    if rc != STITCH_OK:
        m = lib().stitch_batch_last_error(b)
        raise StitchError(rc, m.decode() if m else "")
    return rc


def stitch_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    out = ctypes.c_void_p()
    _batch_check(lib().stitch_batch_create(arr, len(ctxs), ctypes.byref(out)), None)
    return out


def stitch_batch_sequence(b, n_frames, frames, flows_ij, flows_ji, panos, stream=None) -> int:
    """Flat, frame-major pointer lists (see include/stitch.h)."""
    return _batch_check(lib().stitch_batch_sequence(b, n_frames, _ptrs(frames), _ptrs(flows_ij), _ptrs(flows_ji),
                                                    _ptrs(panos), _stream(stream)), b)


def stitch_batch_autotune(b, frames, flows_ij, flows_ji, panos, reps: int = 5):
    """Per-rig tile shapes of the batch, tuned one rig at a time on one frame
    (panos: one panorama per rig). Returns (shapes [n_rigs], ms [n_rigs, 4])."""
    n = len(panos)
    ms = np.zeros(n * STITCH_TILE_SHAPES, dtype=np.float32)
    shapes = np.zeros(n, dtype=np.int32)
    _batch_check(lib().stitch_batch_autotune(b, _ptrs(frames), _ptrs(flows_ij), _ptrs(flows_ji), _ptrs(panos), reps,
                                             shapes.ctypes.data, ms.ctypes.data), b)
    return [int(x) for x in shapes], ms.reshape(n, STITCH_TILE_SHAPES)


def stitch_batch_tile_shapes(b):
    """The batch's tile shape index of every rig."""
    buf = np.zeros(STITCH_BATCH_MAX_RIGS, dtype=np.int32)
    n = lib().stitch_batch_tile_shapes(b, buf.ctypes.data)
    _batch_check(min(n, 0), b)
    return [int(x) for x in buf[:n]]


def stitch_selftest_wait(arrive: bool, limit: int = 1 << 16) -> int:
    """Status of the bounded-wait diagnostic: STITCH_ETIMEOUT without an
    arrival, STITCH_OK with one (no exception either way)."""
    return lib().stitch_selftest_wait(1 if arrive else 0, limit)


def stitch_pair_M_correspondence(ctx, frames, n_pairs: int):
    """One-frame 2D-M of every pair from pixel correspondences (n_pairs, 3, 3)."""
    M = np.zeros((max(n_pairs, 1), 9), dtype=np.float64)
    _check(lib().stitch_pair_M_correspondence(ctx, _ptrs(frames), M.ctypes.data), ctx)
    return M[:n_pairs].reshape(n_pairs, 3, 3)


def stitch_estimate_flow(ctx, frames, flows_ij, flows_ji, stream=None) -> None:
    """Band optical flow of one frame into the caller's float32 [bh, bw, 2]
    device tensors flows_ij / flows_ji (one per pair)."""
    _check(lib().stitch_estimate_flow(ctx, _ptrs(frames), _ptrs(flows_ij), _ptrs(flows_ji), _stream(stream)), ctx)


def stitch_get_flow_luma(ctx, pair: int, side: int, level: int) -> np.ndarray:
    """Level `level` of the luminance pyramid (uint8 [h, w]) of camera
    pair + side over pair `pair`'s band, from the latest stitch_estimate_flow."""
    w, h = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().stitch_get_flow_luma(ctx, pair, side, level, None, ctypes.byref(w), ctypes.byref(h)), ctx)
    out = np.empty((h.value, w.value), dtype=np.uint8)
    _check(lib().stitch_get_flow_luma(ctx, pair, side, level, out.ctypes.data, None, None), ctx)
    return out


def stitch_refine_homographies(ctx, flows_ij, flows_ji, n_cams: int):
    """Refined camera -> panorama homographies (n_cams, 3, 3) and the per-pair
    correction parameters (n_cams - 1, 4) = (t_x, t_y, s_x, s_y) from one
    frame's band flows (device tensors, as for stitch_frame)."""
    H = np.zeros((n_cams, 9), dtype=np.float64)
    prm = np.zeros((max(n_cams - 1, 1), 4), dtype=np.float64)
    _check(lib().stitch_refine_homographies(ctx, _ptrs(flows_ij), _ptrs(flows_ji), prm.ctypes.data, H.ctypes.data),
           ctx)
    return H.reshape(n_cams, 3, 3), prm[:n_cams - 1]


def stitch_batch_destroy(b) -> None:
    if b is not None and b.value:
        lib().stitch_batch_destroy(b)


def stitch_n_pairs(ctx) -> int:
    return lib().stitch_n_pairs(ctx)


def stitch_get_output_hist(ctx) -> np.ndarray:
    """(3, 256) uint32 pre-balance histogram of the latest stitched frame
    (contexts with STITCH_BALANCE_OUTPUT)."""
    h = np.zeros((3, 256), dtype=np.uint32)
    _check(lib().stitch_get_output_hist(ctx, h.ctypes.data), ctx)
    return h


def stitch_window_fallbacks(ctx, reset: bool = False) -> int:
    """Fuse / pre-warp tiles whose source window did not fit in shared memory."""
    n = ctypes.c_ulonglong(0)
    _check(lib().stitch_window_fallbacks(ctx, ctypes.byref(n), 1 if reset else 0), ctx)
    return int(n.value)


def stitch_last_error(ctx=None) -> str:
    m = lib().stitch_last_error(ctx)
    return m.decode() if m else ""


def stitch_destroy(ctx) -> None:
    if ctx is not None and ctx.value:
        lib().stitch_destroy(ctx)


class Stitcher:
    """Convenience owner of a context: frames and flows are torch CUDA tensors."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self.ctx = stitch_init(cfg)
        self.n_cams = cfg.n_cams
        self.n_pairs = cfg.n_cams - 1
        self.bands, self.rects = stitch_get_bands(self.ctx, self.n_pairs)

    def new_pano(self, device="cuda"):
        import torch
        return torch.zeros((3, self.cfg.pano_h, self.cfg.pitch), dtype=torch.uint8, device=device)

    def estimate_color(self, frames, stream=None):
        return stitch_estimate_color(self.ctx, frames, stream)

    def frame(self, frames, flows_ij, flows_ji, pano=None, stream=None):
        if pano is None:
            pano = self.new_pano(frames[0].device)
        stitch_frame(self.ctx, frames, flows_ij, flows_ji, pano, stream)
        return pano

    def color(self):
        return stitch_get_color(self.ctx, self.n_cams)

    def close(self):
        if self.ctx is not None:
            stitch_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        # Never call into CUDA while the interpreter shuts down: the CUDA
        # runtime may already be torn down by then.
        if sys is None or sys.is_finalizing():
            return
        try:
            if getattr(self, "ctx", None) is not None:
                self.close()
        except Exception:
            pass
