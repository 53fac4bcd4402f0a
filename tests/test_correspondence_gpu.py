"""GPU parity of the one-frame colour transfer from pixel correspondences
(stitch_pair_M_correspondence; the 2D-M comparison of Tables 2-3) against
the oracle (oracle/correspondence.py): every pair's M within the colour
matrices' 1e-4 relative bar (the GPU's float32 pre-warp against the oracle's
float64 one, both summed in float64)."""
import numpy as np
import pytest

from oracle.correspondence import pair_M
from paper_2308_09209_b300 import stitch as S

from gpu_common import M_REL_TOL, Pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("config,seed", [("2x640x360", 0), ("3x1920x1080", 2), ("4x640x360cyl", 1)])
def test_correspondence_M_matches_the_oracle(config, seed):
    pr = Pair(config, seed=seed)
    frames, _, _ = pr.inputs(1)
    n = len(pr.rig.cam_w)
    T0 = S.stitch_get_color(pr.st.ctx, n)[3]
    M = S.stitch_pair_M_correspondence(pr.st.ctx, frames, n - 1)
    Mo = pair_M([f.cpu().numpy() for f in frames], pr.oracle.geom)
    for p in range(n - 1):
        assert np.linalg.norm(M[p] - Mo[p]) <= M_REL_TOL * np.linalg.norm(Mo[p]), (p, M[p], Mo[p])
    assert S.stitch_get_color(pr.st.ctx, n)[3] == T0          # the colour state is untouched
    pr.st.close()
