"""Smooth synthetic flow fields for the overlap bands.

A flow field is a float32 [band_h, band_w, 2] array (dx, dy) in panorama
pixels, a sum of four low-frequency plane waves per component whose phases
drift with the frame index t. Components are scaled so that |dx|, |dy| and
the vector length stay within max_flow; near the band's top and bottom rows
the field tapers smoothly to zero. The band size comes from the caller: this
module does not compute any geometry.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def smooth_flow(band_h: int, band_w: int, max_flow: float, seed: int = 0, t: int = 0,
                device="cpu", taper_rows: float = 0.08) -> torch.Tensor:
    rng = np.random.RandomState(seed + 104729)
    y = torch.arange(band_h, dtype=torch.float32, device=device)[:, None]
    x = torch.arange(band_w, dtype=torch.float32, device=device)[None, :]
    out = torch.zeros((band_h, band_w, 2), dtype=torch.float32, device=device)
    for comp in range(2):
        amps = rng.uniform(0.3, 1.0, 4)
        amps = amps / amps.sum()
        for a in amps:
            lam = rng.uniform(80.0, 400.0)
            ang = rng.uniform(0, 2 * math.pi)
            ph = rng.uniform(0, 2 * math.pi)
            spd = rng.uniform(0.05, 0.3)
            kx = math.cos(ang) * 2 * math.pi / lam
            ky = math.sin(ang) * 2 * math.pi / lam
            out[..., comp] += float(a) * torch.sin(kx * x + ky * y + (ph + spd * t))
    out *= float(max_flow) / math.sqrt(2.0) * 0.999
    if taper_rows > 0 and band_h > 4:
        n = max(1.0, taper_rows * band_h)
        d = torch.minimum(y, (band_h - 1) - y) / n
        d = d.clamp(0.0, 1.0)
        wgt = d * d * (3 - 2 * d)
        out *= wgt[..., None]
    return out
