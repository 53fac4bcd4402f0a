"""The one-frame colour transfer from pixel correspondences that the paper
compares its 3D-M against in Tables 2-3 (the 2D-M method of Tian, cited in
section 1 and section 4).

TEST INFRASTRUCTURE ONLY (see the package header): the CUDA path never
imports this module.

Reading: for a pair with colour source i and target j (oriented toward the
reference camera as everywhere else), the corresponding pixels are the two
cameras' pre-warped samples at the same panorama position over the pair's
blend band (the correspondence the homographies give). With X the band's
samples of i and Y those of j as rows of RGB values, the least-squares map
Y ~ X M (row vectors, as Eq. 4) is M = (X^T X)^-1 (X^T Y), in float64."""
import numpy as np

from .flow import band_prewarp


def pair_sums(frames, geom, p):
    """(A = X^T X, B = X^T Y) of pair p over its band, float64 3 x 3 each."""
    i, j = geom.pairs[p]
    band = geom.bands[p]
    X = band_prewarp(np.asarray(frames[i]), geom, i, band).reshape(-1, 3)
    Y = band_prewarp(np.asarray(frames[j]), geom, j, band).reshape(-1, 3)
    return X.T @ X, X.T @ Y


def solve(A, B):
    """M = A^-1 B, float64 (the normal equations' solution)."""
    return np.linalg.solve(A, B)


def pair_M(frames, geom):
    """M of every pair (n_pairs, 3, 3)."""
    return np.stack([solve(*pair_sums(frames, geom, p)) for p in range(len(geom.bands))])
