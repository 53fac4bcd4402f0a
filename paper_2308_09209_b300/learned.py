"""Training and evaluation driver of the learned colour estimator.

Every step of the arithmetic runs in the library's kernels: the plain fit
that labels the pairs (stitch_pairs_label), the network's forward pass, loss,
backward pass and Adam (stitch_mlp_train_step). This module only moves tensors
and picks batches.

    python -m paper_2308_09209_b300.learned --pairs 200000 --epochs 8 --out weights.npz

draws the seeded training pairs (synthetic scenes under random gain, gamma,
offset and colour cast), labels them on the GPU, trains, and writes the
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


def main():
    from synth import make_pairs
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=200000)
    ap.add_argument("--held-out", type=int, default=8192)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    S.stitch_mlp_n_params()
    t0 = time.perf_counter()
    pairs, _ = make_pairs(a.pairs + a.held_out, seed=a.seed, device="cuda")
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
    print(json.dumps(rep))
    net.close()


if __name__ == "__main__":
    main()
