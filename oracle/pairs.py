"""Labels and features of independent overlap pairs (the training data of the
learned estimator), plain FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

For one pair (a patch of side i and a patch of side j, packed RGB) the label
is the one-frame plain fit of section 2.1: histograms (step 2), the
specification LUT (step 3), A = I_i^T I_i and B = I_i^T L(I_i), M = A^-1 B
(Eq. 3, float64; an ill-conditioned A or an empty side gives I and a flag),
plus, per channel, the span (m2 - m1) / 255 of the lambda-quantile knots
(section 2.2) of the two patches' pooled histogram.

Features: each side's three channel histograms scaled by 256 / pixel count,
side i first, channel-major, rounded to bfloat16.
"""
from __future__ import annotations

import numpy as np

from . import balance, color
from .mlp import round_bf16


def label(patch_i, patch_j, lam=0.05):
    """(features[1536] float64 of bfloat16 values, targets[12] float64,
    M[3,3] float64, flag int) of one pair."""
    pi = np.asarray(patch_i).reshape(-1, 3)
    pj = np.asarray(patch_j).reshape(-1, 3)
    Hi = color.channel_histograms(pi)
    Hj = color.channel_histograms(pj)
    lut = color.spec_lut(Hi, Hj)
    A, B = color.normal_equations(pi, lut)
    M, ok = color.solve_transfer(A, B)
    ok = ok and pi.shape[0] > 0 and pj.shape[0] > 0
    if not ok:
        M = np.eye(3)
    m1, m2 = balance.knots(Hi + Hj, lam)
    s = (m2 - m1).astype(np.float64) / 255.0
    ni, nj = pi.shape[0], pj.shape[0]
    fi = (Hi.reshape(-1) * 256.0) / ni if ni else np.zeros(768)
    fj = (Hj.reshape(-1) * 256.0) / nj if nj else np.zeros(768)
    feat = round_bf16(np.concatenate([fi, fj]))
    targ = np.concatenate([(M - np.eye(3)).reshape(-1), s])
    return feat, targ, M, 0 if ok else 1
