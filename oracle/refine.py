"""Homography refinement from the blend-band flows (section 3.1, Eq. 13-14).

TEST INFRASTRUCTURE ONLY (see the package header): the CUDA path never
imports this module.

The paper revises each camera's homography with a skew (translation) matrix
and a scale matrix whose parameters come from SURF matches in a widened
overlap region (Eq. 13), H' = M H N (Eq. 14). Here the matches are the flow
fields the path already takes as inputs (section 3.2), and the parameters are
robust statistics of those fields over each pair's blend band:

* flow_ij is sampled for the pair's left camera: its pre-warped content at
  q + flow_ij(q) shows what the right camera shows at q; flow_ji is the same
  for the right camera. So the left content sits displaced by about d =
  (median(flow_ij) - median(flow_ji)) / 2 against the right content, and its
  displacement grows across the band by about g = (median of the forward
  differences of flow_ij - the same of flow_ji) / 2 per pixel (x differences
  of the x component, y differences of the y component).
* A median is the ((n - 1) // 2)-th smallest of the finite values (an element,
  no averaging); the forward differences are float32 subtractions of
  neighbouring float32 samples, kept where the difference is finite. With no
  finite value the statistic is 0.
* The camera of the pair farther from the reference camera is moved onto its
  neighbour: in panorama pixels, q -> c + s (q - c) + t about the band centre
  c = ((x0 + x1 - 1) / 2, (y0 + y1 - 1) / 2), with (t, s) = (-d, 1 - g) when
  that camera is the left one and (+d, 1 + g) when it is the right one. This
  is the M N pair of Eq. 13 (translation after a scale), applied on the
  panorama side of the camera -> panorama homography and centred on the band
  (reading: the paper's N acts on image coordinates about the image origin,
  where a scale error would also shift the band).
* Corrections compose outward from the reference camera (which keeps its
  homography): C_ref = I, C_k = C_(k+1) A_k to its left, C_k = C_(k-1) A_(k-1)
  to its right, and H'_k = C_k H_k.

Planar panoramas only (a cylinder's panorama pixels are not a projective
image of the camera plane)."""
import numpy as np


def lower_median(values):
    """The ((n - 1) // 2)-th smallest element of the finite entries of
    ``values`` (brute force: a full sort); 0.0 when there is none."""
    v = np.asarray(values).ravel()
    v = v[np.isfinite(v)]
    if v.size == 0:
        return 0.0
    return float(np.sort(v, kind="stable")[(v.size - 1) // 2])


def flow_stats(flow):
    """(median x, median y, median x-difference of x, median y-difference of
    y) of one band flow field, float32 (bh, bw, 2)."""
    f = np.asarray(flow, dtype=np.float32)
    fx, fy = f[..., 0], f[..., 1]
    with np.errstate(invalid="ignore", over="ignore"):
        ddx = (fx[:, 1:] - fx[:, :-1]).astype(np.float32)   # float32 subtraction
        ddy = (fy[1:, :] - fy[:-1, :]).astype(np.float32)
    return lower_median(fx), lower_median(fy), lower_median(ddx), lower_median(ddy)


def pair_params(geom, p, flow_ij, flow_ji):
    """(t_x, t_y, s_x, s_y) of the correction of pair p's outer camera, and
    that correction as a 3x3 matrix in panorama pixels."""
    a = flow_stats(flow_ij)
    b = flow_stats(flow_ji)
    d = ((a[0] - b[0]) / 2.0, (a[1] - b[1]) / 2.0)
    g = ((a[2] - b[2]) / 2.0, (a[3] - b[3]) / 2.0)
    sign = -1.0 if p < geom.ref else 1.0          # left camera outer <=> p + 1 <= ref
    t = (sign * d[0], sign * d[1])
    s = (1.0 + sign * g[0], 1.0 + sign * g[1])
    x0, x1, y0, y1 = geom.bands[p]
    cx, cy = (x0 + x1 - 1) / 2.0, (y0 + y1 - 1) / 2.0
    M = np.array([[1.0, 0.0, t[0]], [0.0, 1.0, t[1]], [0.0, 0.0, 1.0]])     # Eq. 13, skew (translation)
    N = np.array([[s[0], 0.0, cx - s[0] * cx], [0.0, s[1], cy - s[1] * cy], [0.0, 0.0, 1.0]])  # scale about c
    return (t[0], t[1], s[0], s[1]), M @ N


def refine(geom, H, flows_ij, flows_ji):
    """Refined camera -> panorama homographies (n, 3, 3) and the per-pair
    parameters (n - 1, 4) from one frame's band flows."""
    n = len(H)
    params = np.zeros((n - 1, 4))
    A = []
    for p in range(n - 1):
        prm, Ap = pair_params(geom, p, flows_ij[p], flows_ji[p])
        params[p] = prm
        A.append(Ap)
    C = [None] * n
    C[geom.ref] = np.eye(3)
    for k in range(geom.ref - 1, -1, -1):
        C[k] = C[k + 1] @ A[k]
    for k in range(geom.ref + 1, n):
        C[k] = C[k - 1] @ A[k - 1]
    Hn = np.stack([C[k] @ np.asarray(H[k], dtype=np.float64) for k in range(n)])
    return Hn, params
