"""GPU parity of the homography refinement from the band flows
(stitch_refine_homographies; section 3.1, Eq. 13-14) against the oracle
(oracle/refine.py): the per-pair parameters bit for bit (exact medians by
radix selection), the refined homographies to float64 rounding, known
translations put back, and argument errors."""
import numpy as np
import pytest
import torch

from oracle.refine import refine
from paper_2308_09209_b300 import stitch as S

from gpu_common import Pair, ensure_built

pytestmark = pytest.mark.gpu


def _H_close(a, b):
    for k in range(len(a)):
        assert np.allclose(a[k], b[k], rtol=0, atol=1e-12 * np.abs(b[k]).max()), k


@pytest.mark.parametrize("config,seed", [("2x640x360", 0), ("3x1920x1080", 2), ("4x1920x1080", 1)])
def test_refinement_matches_the_oracle(config, seed):
    pr = Pair(config, seed=seed)
    _, fij, fji = pr.inputs(0)
    # non-finite samples are skipped by both sides
    fij[0].view(-1)[::997] = float("nan")
    fji[-1][3, :, 1] = float("inf")
    n = len(pr.rig.cam_w)
    H, prm = S.stitch_refine_homographies(pr.st.ctx, fij, fji, n)
    Ho, prmo = refine(pr.oracle.geom, [np.asarray(h, np.float64).reshape(3, 3) for h in pr.rig.H],
                      [f.cpu().numpy() for f in fij], [f.cpu().numpy() for f in fji])
    assert np.array_equal(prm, prmo), (prm, prmo)
    _H_close(H, Ho)
    # the context is unchanged: a second call gives the same
    H2, prm2 = S.stitch_refine_homographies(pr.st.ctx, fij, fji, n)
    assert np.array_equal(prm2, prm) and np.array_equal(H2, H)
    pr.st.close()


def test_known_translations_are_put_back():
    """Three cameras, reference 1: the left camera's content sits at +d0
    against the middle one and the right camera's at +d2; constant flows say
    so, and the refinement moves the outer cameras by -d0 and -d2."""
    pr = Pair("3x1920x1080", seed=4)
    bands = pr.st.bands.tolist()
    d0, d2 = (2.5, -0.75), (-1.25, 1.5)

    def const(p, v):
        x0, x1, y0, y1 = bands[p]
        f = torch.empty((y1 - y0, x1 - x0, 2), dtype=torch.float32, device="cuda")
        f[..., 0], f[..., 1] = v
        return f

    fij = [const(0, d0), const(1, (-d2[0], -d2[1]))]
    fji = [const(0, (-d0[0], -d0[1])), const(1, d2)]
    H, prm = S.stitch_refine_homographies(pr.st.ctx, fij, fji, 3)
    assert prm.tolist() == [[-2.5, 0.75, 1.0, 1.0], [1.25, -1.5, 1.0, 1.0]]
    H0 = [np.asarray(h, np.float64).reshape(3, 3) for h in pr.rig.H]
    T = lambda dx, dy: np.array([[1.0, 0.0, dx], [0.0, 1.0, dy], [0.0, 0.0, 1.0]])  # noqa: E731
    assert np.array_equal(H[1], H0[1])
    _H_close(H, [T(-d0[0], -d0[1]) @ H0[0], H0[1], T(-d2[0], -d2[1]) @ H0[2]])
    pr.st.close()


def test_refinement_argument_errors():
    ensure_built()
    pr = Pair("2x640x360", seed=0)
    _, fij, fji = pr.inputs(0)
    with pytest.raises(S.StitchError):
        S.stitch_refine_homographies(pr.st.ctx, [0], fji, 2)
    bad = torch.empty(fij[0].numel() * 4 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.StitchError):
        S.stitch_refine_homographies(pr.st.ctx, [bad.data_ptr() + 4], fji, 2)   # not 8-byte aligned
    pr.st.close()
    cyl = Pair("4x640x360cyl", seed=0)
    _, fij, fji = cyl.inputs(0)
    with pytest.raises(S.StitchError):
        S.stitch_refine_homographies(cyl.st.ctx, fij, fji, 4)
    cyl.st.close()
