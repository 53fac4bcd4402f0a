"""3D-M colour transfer, float64 / int64 (paper section 2.1, Eq. 1-4).

Per adjacent pair the paper (section 2.1):
  step 2  takes the histograms G_i, G_j of the overlap region in frames i, j;
  step 3  specifies G_i onto G_j (j is the reference), giving the revised
          image i;
  step 4  fits M = [I_i^T I_i]^-1 I_i^T I_j (Eq. 1) where I_i holds the pixels
          of image i and I_j those of the revised image i, stacking frames
          T, T-1, T-2 on top of each other (Eq. 2-3);
  step 5  corrects image i as I'_i = I_i . M (Eq. 4), row-vector convention.

Readings (the printed Eq. 3 has garbled transposes): with Eq. 2's (3n x 3)
stacking, Eq. 3 is the normal equations of the stacked system, so
A = sum_t I_ti^T I_ti and B = sum_t I_ti^T I_tj over the frames of the
window, and M = A^-1 B. The window holds the last W frames (W = 3 in the
paper) that exist, extending the first-frames rule of section 2.2 to M.
"""
from __future__ import annotations

import numpy as np

COND_LIMIT = 1e12


def channel_histograms(pix: np.ndarray) -> np.ndarray:
    """Per-channel 256-bin histograms of an (n, 3) uint8 pixel list (step 2)."""
    pix = np.asarray(pix).reshape(-1, 3)
    return np.stack([np.bincount(pix[:, c].astype(np.int64), minlength=256) for c in range(3)])


def spec_lut(hist_i: np.ndarray, hist_j: np.ndarray) -> np.ndarray:
    """Histogram specification of G_i onto G_j (step 3, Fig. 2).

    For every level v of image i, L(v) is the smallest level u of image j
    whose cumulative share reaches v's cumulative share:
        CDF_j(u) / n_j >= CDF_i(v) / n_i,
    evaluated exactly as CDF_j(u) * n_i >= CDF_i(v) * n_j in integers.
    Returns (3, 256) int64; rows with an empty side are the identity."""
    lut = np.zeros((3, 256), dtype=np.int64)
    for c in range(3):
        hi = np.asarray(hist_i[c], dtype=np.int64)
        hj = np.asarray(hist_j[c], dtype=np.int64)
        ni, nj = int(hi.sum()), int(hj.sum())
        if ni == 0 or nj == 0:
            lut[c] = np.arange(256)
            continue
        cdf_i = np.cumsum(hi)
        cdf_j = np.cumsum(hj)
        for v in range(256):
            need = int(cdf_i[v]) * nj
            u = 0
            while int(cdf_j[u]) * ni < need:
                u += 1
            lut[c, v] = u
    return lut


def revised_image(pix_i: np.ndarray, lut: np.ndarray) -> np.ndarray:
    """The revised image i: each channel of image i mapped through its LUT (step 3)."""
    pix_i = np.asarray(pix_i).reshape(-1, 3).astype(np.int64)
    return np.stack([lut[c][pix_i[:, c]] for c in range(3)], 1)


def normal_equations(pix_i: np.ndarray, lut: np.ndarray):
    """One frame's A_t = I_i^T I_i and B_t = I_i^T I_j (Eq. 1 / Eq. 3 terms), int64."""
    X = np.asarray(pix_i).reshape(-1, 3).astype(np.int64)
    Y = revised_image(X, lut)
    return X.T @ X, X.T @ Y


def solve_transfer(A: np.ndarray, B: np.ndarray):
    """M = A^-1 B in float64 (Eq. 1 / Eq. 3). Returns (M, ok); ok is False when
    the 1-norm condition number of A exceeds 1e12 (e.g. a flat overlap)."""
    Af = np.asarray(A, dtype=np.float64)
    Bf = np.asarray(B, dtype=np.float64)
    with np.errstate(all="ignore"):
        try:
            cond = np.linalg.cond(Af, 1)
        except np.linalg.LinAlgError:
            cond = np.inf
    if not np.isfinite(cond) or cond > COND_LIMIT:
        return None, False
    return np.linalg.solve(Af, Bf), True


def chain_to_reference(M_pairs, pairs, ref: int, n_cams: int) -> np.ndarray:
    """Composite per-camera matrix into the reference camera's colours.

    Pair p moves camera i's colours to its neighbour j (one step toward the
    reference). With the row-vector convention of Eq. 4, camera k's composite
    is M_k = M_(k->nb) . M_nb and the reference keeps the identity."""
    out = [None] * n_cams
    out[ref] = np.eye(3)
    for k in range(ref - 1, -1, -1):
        p = k                       # pair (k, k+1), i = k, j = k + 1
        assert pairs[p] == (k, k + 1)
        out[k] = M_pairs[p] @ out[k + 1]
    for k in range(ref + 1, n_cams):
        p = k - 1                   # pair (k-1, k), i = k, j = k - 1
        assert pairs[p] == (k, k - 1)
        out[k] = M_pairs[p] @ out[k - 1]
    return np.stack(out)
