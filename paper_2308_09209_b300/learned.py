"""Training and evaluation driver of the learned colour estimator.

Every step of the arithmetic runs in the library's kernels: the plain fit
that labels the pairs (stitch_pairs_label), the network's forward pass, loss,
backward pass and Adam (stitch_mlp_train_step). This module only moves tensors
and picks batches.

    python -m paper_2308_09209_b300.learned --pairs 200000 --epochs 40 --out weights.npz --evaluate

draws the seeded training pairs (synthetic scenes under random gain, gamma,
offset and colour cast, each side three frames of a moving scene like a rig's
window-pooled overlap), labels them on the GPU, trains, and writes the
float32 parameters and the target normalisation to ``--out``.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import stitch as S


def label_pairs(pairs: torch.Tensor, lam: float = 0.05, chunk: int = 65536):
    """Plain one-frame fit of every pair (uint8 CUDA tensor [n, 2, ph, pw, 3]):
    (features bfloat16 bits int16 [n, 1536], targets float32 [n, 12],
    M float64 [n, 9], flags int32 [n]), all on the GPU."""
    n, _, ph, pw, _ = pairs.shape
    dev = pairs.device
    feat = torch.empty((n, S.STITCH_MLP_IN), dtype=torch.int16, device=dev)
    targ = torch.empty((n, S.STITCH_MLP_OUT), dtype=torch.float32, device=dev)
    M = torch.empty((n, 9), dtype=torch.float64, device=dev)
    flags = torch.empty((n,), dtype=torch.int32, device=dev)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        S.stitch_pairs_label(pairs[c0:c1], c1 - c0, pw, ph, lam, feat[c0:c1], targ[c0:c1], M[c0:c1], flags[c0:c1])
    torch.cuda.synchronize(dev)
    return feat, targ, M, flags


def target_norm(targ: torch.Tensor):
    """Per-output mean and standard deviation of the training targets."""
    t = targ.double()
    mu = t.mean(0).float().cpu().numpy()
    sd = t.std(0).clamp_min(1e-6).float().cpu().numpy()
    return mu, sd


def train(feat, targ, epochs=8, batch=512, lr=1e-3, lr_min=1e-5, seed=0, mask=None, log=None):
    """Train a new network on (features, targets) with a cosine learning-rate
    schedule. Returns (Mlp, per-epoch mean loss list)."""
    n = feat.shape[0]
    if mask is not None:
        keep = torch.nonzero(mask).flatten()
        feat, targ = feat[keep], targ[keep]
        n = feat.shape[0]
    batch = max(32, (min(batch, n) // 32) * 32)
    net = S.Mlp(max_batch=batch, seed=seed)
    mu, sd = target_norm(targ)
    S.stitch_mlp_set_norm(net.h, mu, sd)
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps_per_epoch = n // batch
    total = steps_per_epoch * epochs
    loss = torch.zeros(steps_per_epoch, dtype=torch.float32, device=feat.device)
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(feat.device)
        for k in range(steps_per_epoch):
            idx = perm[k * batch:(k + 1) * batch]
            xb = feat.index_select(0, idx).contiguous()
            tb = targ.index_select(0, idx).contiguous()
            cur = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / max(1, total)))
            S.stitch_mlp_train_step(net.h, xb, tb, batch, cur, loss[k:k + 1])
            step += 1
        hist.append(float(loss.mean().item()))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f}")
    return net, hist


def predict(net, feat: torch.Tensor, chunk: int = None) -> torch.Tensor:
    """Network output (target units) for every row of feat."""
    n = feat.shape[0]
    chunk = chunk or net.max_batch
    y = torch.empty((n, S.STITCH_MLP_OUT), dtype=torch.float32, device=feat.device)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        S.stitch_mlp_forward(net.h, feat[c0:c1].contiguous(), c1 - c0, y[c0:c1])
    torch.cuda.synchronize(feat.device)
    return y


def save(net, path, mu, sd):
    np.savez(path, params=S.stitch_mlp_get_params(net.h), mu=np.asarray(mu, np.float32),
             sd=np.asarray(sd, np.float32))


def load(path, max_batch=256):
    d = np.load(path)
    net = S.Mlp(max_batch=max_batch, seed=0)
    S.stitch_mlp_set_params(net.h, d["params"])
    S.stitch_mlp_set_norm(net.h, d["mu"], d["sd"])
    return net, d["mu"], d["sd"]


def evaluate_gain(net, config="2x640x360", seeds=(101, 102, 103, 104), n_frames=8, objects=6):
    """Learned against plain colour estimate on held-out synthetic rigs with a
    known photometric response per camera.

    For every frame and pair (i -> j) the true transfer is the least-squares
    3x3 map from camera i's pixels to what camera j's response gives for the
    same scene colours over camera i's whole frame; a matrix's error is the RMS
    colour error (grey levels) of that map applied with the matrix instead.
    Reported per estimator: the mean error, the frame-to-frame standard
    deviation of M (mean over entries, frames after the window fills), and the
    estimate's GPU time per frame; plus the learned path's fallback rate.
    ``objects`` moving objects make the frames (and so M) change over time."""
    from synth import Scene, render_camera_frames, rig_for_config
    from synth.scene import _photometric
    res = {k: dict(err=[], M=[]) for k in ("plain", "learned_raw", "learned_used", "truth")}
    t_plain, t_learned, n_l, n_f = 0.0, 0.0, 0, 0
    n_est = 0
    for seed in seeds:
        rig, seq = rig_for_config(config, seed=seed, **({} if objects is None else {"objects": objects}))
        scene = Scene(rig.pano_w, rig.pano_h, n_objects=seq.get("objects", 0), seed=seed)
        base = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                        max_flow=seq["max_flow"], flags=0)
        lcfg = S.Config(rig.cam_w, rig.cam_h, rig.H, rig.pano_w, rig.pano_h, window=seq["window"],
                        max_flow=seq["max_flow"], flags=S.STITCH_LEARNED)
        sp, sl = S.Stitcher(base), S.Stitcher(lcfg)
        S.stitch_attach_mlp(sl.ctx, net.h)
        S.stitch_profile(sp.ctx, True)
        S.stitch_profile(sl.ctx, True)
        npair = rig.n_cams - 1
        per = {k: [] for k in res}
        for t in range(n_frames):
            frames = render_camera_frames(rig, scene, t, device="cuda")
            sp.estimate_color(frames)
            sl.estimate_color(frames)
            Mp = S.stitch_get_pair_M(sp.ctx, npair)
            Mh, r, used = S.stitch_get_learned(sl.ctx, npair)
            Mu = S.stitch_get_pair_M(sl.ctx, npair)
            mats = dict(plain=Mp, learned_raw=Mh, learned_used=Mu)
            truth = []
            for p in range(npair):
                i = p if p < rig.n_cams // 2 else p + 1          # colour source of pair p
                j = p + 1 if p < rig.n_cams // 2 else p          # its neighbour toward the reference
                w, h = rig.cam_w[i], rig.cam_h[i]
                G = torch.tensor(rig.G[i], dtype=torch.float64, device="cuda")
                v, u = torch.meshgrid(torch.arange(0, h, 4, dtype=torch.float64, device="cuda"),
                                      torch.arange(0, w, 4, dtype=torch.float64, device="cuda"), indexing="ij")
                den = G[2, 0] * u + G[2, 1] * v + G[2, 2]
                X = ((G[0, 0] * u + G[0, 1] * v + G[0, 2]) / den).float()
                Y = ((G[1, 0] * u + G[1, 1] * v + G[1, 2]) / den).float()
                sc = scene.render(X, Y, t)
                xi = _photometric(sc, rig.gain[i], rig.gamma[i], rig.offset[i], rig.cast[i]).reshape(-1, 3).double()
                yj = _photometric(sc, rig.gain[j], rig.gamma[j], rig.offset[j], rig.cast[j]).reshape(-1, 3).double()
                Mt = torch.linalg.lstsq(xi, yj).solution
                truth.append(Mt.cpu().numpy())
                for k, Ms in list(mats.items()) + [("truth", None)]:
                    Mk = Mt if Ms is None else torch.tensor(Ms[p], dtype=torch.float64, device="cuda")
                    e = float((xi @ Mk - yj).pow(2).sum(1).mean().sqrt())
                    per[k].append((t, p, e, (Mk.cpu().numpy() if Ms is None else Ms[p]).copy()))
        pr_p = S.stitch_profile_read(sp.ctx)
        pr_l = S.stitch_profile_read(sl.ctx)
        t_plain += pr_p["estimate_ms"]
        t_learned += pr_l["estimate_ms"]
        n_est += pr_p["estimate_n"]
        a, b = S.stitch_learned_stats(sl.ctx)
        n_l += a
        n_f += b
        for k in res:
            res[k]["err"] += [e for (_, _, e, _) in per[k]]
            for p in range(npair):
                Ms = np.stack([M for (t, pp, _, M) in per[k] if pp == p and t >= seq["window"]])
                res[k]["M"].append(float(Ms.std(axis=0).mean()) if len(Ms) > 1 else 0.0)
        sp.close()
        sl.close()
    out = {k: dict(rms_colour_error=float(np.mean(v["err"])), sigma_M=float(np.mean(v["M"]))) for k, v in res.items()}
    out["plain"]["estimate_ms_per_frame"] = t_plain / max(n_est, 1)
    out["learned_used"]["estimate_ms_per_frame"] = t_learned / max(n_est, 1)
    out["estimate_timing"] = ("GPU time between the stage events around each direct stitch_estimate_color call "
                              "(one call per frame, so the gaps while the host launches the next kernel count: "
                              "2 launches for the plain estimate, 8 for the learned one)")
    out["fallback_rate"] = n_f / max(n_l + n_f, 1)
    out["rigs"] = f"{len(seeds)} x {config}, {n_frames} frames each"
    return out


def main():
    from synth import make_window_pairs
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=200000)
    ap.add_argument("--held-out", type=int, default=8192)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--evaluate", action="store_true", help="also run the learned-vs-plain evaluation")
    a = ap.parse_args()
    S.stitch_mlp_n_params()
    t0 = time.perf_counter()
    pairs, _ = make_window_pairs(a.pairs + a.held_out, seed=a.seed, device="cuda")
    t1 = time.perf_counter()
    feat, targ, M, flags = label_pairs(pairs)
    t2 = time.perf_counter()
    n = a.pairs
    ok = flags[:n] == 0
    net, hist = train(feat[:n], targ[:n], epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed, mask=ok,
                      log=lambda s: print(s, flush=True))
    t3 = time.perf_counter()
    y = predict(net, feat[n:])
    err = (y - targ[n:]).double()
    rep = dict(pairs=n, held_out=a.held_out, epochs=a.epochs, generate_s=t1 - t0, label_s=t2 - t1, train_s=t3 - t2,
               loss=hist, held_out_rmse_M=float(err[:, :9].pow(2).mean().sqrt()),
               held_out_rmse_span=float(err[:, 9:].pow(2).mean().sqrt()),
               label_flagged=int((flags != 0).sum()))
    if a.out:
        mu, sd = target_norm(targ[:n][ok])
        save(net, a.out, mu, sd)
    if a.evaluate:
        rep["gain"] = evaluate_gain(net)
    print(json.dumps(rep))
    net.close()


if __name__ == "__main__":
    main()
