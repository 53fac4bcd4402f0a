"""Per-frame sequence of the stitching method with its temporal state, float64.

The order follows the paper's system (section 4: geometric warping, colour
correction, local warping, fusion) with the colour statistics of frame T
taken before frame T is fused:

  estimate_color(frames_T):
    for every adjacent pair, histograms of the overlap in both frames
    (section 2.1 step 2), specification (step 3), this frame's normal
    equation terms A_T, B_T (Eq. 3), M over the last W frames (Eq. 1-3);
    M chained to the reference camera (Eq. 4); knots m1, m2 of the pooled
    histogram and their 3-frame mean (Eq. 6-7); the balance curve (Eq. 5).
  frame(frames_T, flows_T):
    pre-warp, local warping, fusion, balance (section 3, Eq. 15-18).

If the window's A is ill-conditioned (1-norm condition > 1e12) or a side of
the overlap is empty, the pair keeps its previous M (identity before the
first success) and the frame is flagged singular.

Balance on the stitched image (flag BALANCE_OUTPUT): frame(T) keeps the
histogram of its panorama before the balance (``balance.output_histogram``)
and estimate_color(T + 1) takes the knots from it instead of the pooled raw
histogram; the first frame, with no stitched predecessor, is not balanced.

Learned mode (flag LEARNED with a network given): after the plain estimate,
each pair's features are its window-pooled overlap histograms (side i then
side j, each scaled by 256 / count, bfloat16), the network predicts M_hat - I
(``oracle.mlp``), and the pair takes M_hat when its plain fit succeeded and
r = tr(D^T A D) / tr(M*^T A M*) <= 1e-3 over the window's A, with D = M_hat - M* and
M* the window's plain fit (the relative excess of Eq. 2's least-squares error); otherwise
it keeps the plain result. The chosen matrices are chained as usual.
"""
from __future__ import annotations

import numpy as np

from . import balance as bal
from . import color as col
from . import mlp as _mlp
from .geometry import Geometry
from .warp import stitch as _stitch, fuse_pixels, finish


class OracleStitcher:
    def __init__(self, H, cam_w, cam_h, pano_w, pano_h, ref_cam=None, window=3,
                 lam=0.05, max_flow=8.0, flags=0, mlp=None, projection=0, cyl=None):
        self.geom = Geometry(H, cam_w, cam_h, pano_w, pano_h, ref_cam, projection=projection, cyl=cyl)
        self.window = int(window)
        self.lam = float(lam)
        self.max_flow = float(max_flow)
        self.flags = int(flags)
        self.T = 0
        n_p = self.geom.n - 1
        self.ab_hist = []                      # per frame: list of (A_t, B_t) per pair
        self.knot_hist = []                    # per frame: (m1, m2)
        self.M_pair = [np.eye(3) for _ in range(n_p)]
        self.M_cam = np.tile(np.eye(3), (self.geom.n, 1, 1))
        self.curve = bal.curve_params(np.zeros(3), np.zeros(3), self.lam)
        self.singular = False
        self.last_stats = None
        self.mlp = mlp                         # dict(params, mu, sd) for learned mode
        self.hist_hist = []                    # per frame: list of (Hi, Hj) per pair
        self.learned = None                    # latest (M_hat, r, used) per pair
        self.n_learned = 0
        self.n_fallback = 0
        self.out_hist = None                   # balance on the stitched image: last frame's histogram

    # -- statistics of one frame (section 2.1 steps 2-3, Eq. 3 terms) --------
    def frame_stats(self, frames):
        g = self.geom
        pooled = sum(col.channel_histograms(np.asarray(f).reshape(-1, 3)) for f in frames)
        pairs = []
        for p, (i, j) in enumerate(g.pairs):
            ri = g.rect_of(p, i)
            rj = g.rect_of(p, j)
            pi = np.asarray(frames[i])[ri[2]:ri[3], ri[0]:ri[1]].reshape(-1, 3)
            pj = np.asarray(frames[j])[rj[2]:rj[3], rj[0]:rj[1]].reshape(-1, 3)
            Hi = col.channel_histograms(pi)
            Hj = col.channel_histograms(pj)
            lut = col.spec_lut(Hi, Hj)
            A, B = col.normal_equations(pi, lut)
            pairs.append(dict(Hi=Hi, Hj=Hj, lut=lut, A=A, B=B, n_i=pi.shape[0], n_j=pj.shape[0],
                              pix_i=pi))
        return dict(pooled=pooled, pairs=pairs)

    def estimate_color(self, frames):
        g = self.geom
        st = self.frame_stats(frames)
        self.last_stats = st
        self.ab_hist.append([(pp["A"], pp["B"], pp["n_i"], pp["n_j"]) for pp in st["pairs"]])
        self.hist_hist.append([(pp["Hi"], pp["Hj"]) for pp in st["pairs"]])
        win = self.ab_hist[-self.window:]
        self.singular = False
        ok_p, AB = [], []
        for p in range(g.n - 1):
            A = sum(w[p][0] for w in win)
            B = sum(w[p][1] for w in win)
            empty = any(w[p][2] == 0 or w[p][3] == 0 for w in win)
            M, ok = (None, False) if empty else col.solve_transfer(A, B)
            if ok:
                self.M_pair[p] = M
            else:
                self.singular = True
            ok_p.append(ok)
            AB.append((A, B))
        if (self.flags & 8) and self.mlp is not None and g.n > 1:
            self._learned_select(ok_p, AB)
        self.M_cam = col.chain_to_reference(self.M_pair, g.pairs, g.ref, g.n)
        if self.flags & 16:
            # balance on the stitched image of the previous frame (one-frame lag)
            if self.out_hist is not None and int(self.out_hist[0].sum()) > 0:
                m1, m2 = bal.knots(self.out_hist, self.lam)
                self.knot_hist.append((m1, m2))
                sm1, sm2 = bal.smooth(self.knot_hist)
                self.curve = bal.curve_params(sm1, sm2, self.lam)
            else:
                self.curve = bal.curve_params(np.zeros(3), np.zeros(3), self.lam)
            self.out_hist = None
        else:
            m1, m2 = bal.knots(st["pooled"], self.lam)
            self.knot_hist.append((m1, m2))
            sm1, sm2 = bal.smooth(self.knot_hist)
            self.curve = bal.curve_params(sm1, sm2, self.lam)
        self.T += 1
        return not self.singular

    def learned_features(self):
        """Window-pooled features of every pair, (n_pairs, 1536) float64 of
        bfloat16 values."""
        hw = self.hist_hist[-self.window:]
        rows = []
        for p in range(self.geom.n - 1):
            Hi = sum(np.asarray(h[p][0], dtype=np.int64) for h in hw)
            Hj = sum(np.asarray(h[p][1], dtype=np.int64) for h in hw)
            ni, nj = int(Hi[0].sum()), int(Hj[0].sum())
            fi = (Hi.reshape(-1) * 256.0) / ni if ni else np.zeros(768)
            fj = (Hj.reshape(-1) * 256.0) / nj if nj else np.zeros(768)
            rows.append(np.concatenate([fi, fj]))
        return _mlp.round_bf16(np.stack(rows))

    def _learned_select(self, ok_p, AB):
        X = self.learned_features()
        Y, _ = _mlp.forward(self.mlp["params"], X)
        Y = Y[:, :_mlp.N_OUT] * np.asarray(self.mlp["sd"], dtype=np.float64) + np.asarray(self.mlp["mu"],
                                                                                           dtype=np.float64)
        out = []
        for p, (A, B) in enumerate(AB):
            M_hat = np.eye(3) + Y[p, :9].reshape(3, 3)
            r = _mlp.residual(A, B, M_hat)
            use = bool(ok_p[p] and np.all(np.isfinite(M_hat)) and r <= 1e-3)
            if use:
                self.M_pair[p] = M_hat
                self.n_learned += 1
            else:
                self.n_fallback += 1
            out.append((M_hat, r, use))
        self.learned = out

    def frame(self, frames, flows_ij, flows_ji):
        frames = [np.asarray(f) for f in frames]
        if not (self.flags & 16):
            return _stitch(frames, self.geom, flows_ij, flows_ji, self.M_cam, self.curve,
                           self.max_flow, self.flags)
        cov = np.zeros((self.geom.pano_h, self.geom.pano_w), dtype=bool)
        planes, near, vals = _stitch(frames, self.geom, flows_ij, flows_ji, self.M_cam, self.curve,
                                     self.max_flow, self.flags, cov_out=cov)
        self.out_hist = bal.output_histogram(vals, cov)
        return planes, near, vals

    def pixels(self, frames, flows_ij, flows_ji, xs, ys):
        """Output of selected pixels only: (uint8 (N, 3), near_edge (N,))."""
        frames = [np.asarray(f) for f in frames]
        v, c, e = fuse_pixels(frames, self.geom, flows_ij, flows_ji, self.M_cam, self.max_flow,
                              self.flags, xs, ys)
        return finish(v, c, self.curve, self.flags), e
