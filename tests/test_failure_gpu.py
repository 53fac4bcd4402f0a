"""Failure detection without a GPU fault: the library's bounded device waits
give up and report STITCH_ETIMEOUT, and the device stays usable afterwards
(a frame stitched right after matches the oracle as usual)."""
import pytest

from paper_2308_09209_b300 import stitch as S

from gpu_common import Pair, assert_pano_ok, compare_pano, ensure_built

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    ensure_built()
    assert S.stitch_selftest_wait(False, 1 << 14) == S.STITCH_ETIMEOUT
    assert S.stitch_selftest_wait(True, 1 << 14) == S.STITCH_OK
    assert S.stitch_selftest_wait(False, 0) == S.STITCH_EINVAL
    pr = Pair("2x640x360", seed=1)
    out = pr.step(0)
    assert_pano_ok(compare_pano(out["pano"], out["planes"], out["near"], pr.rig.pano_w))
    pr.st.close()


def test_tensor_core_timeouts_are_reported_and_a_failed_drain_is_sticky():
    """A timed-out wait (bit 0) is reported once; a failed drain (bit 2) keeps
    the tcgen05 engine refused, while the mma.sync engine keeps working."""
    import torch
    ensure_built()
    import numpy as np
    mlp = S.stitch_mlp_create(64, 3)
    S.stitch_mlp_set_norm(mlp, np.zeros(S.STITCH_MLP_OUT), np.ones(S.STITCH_MLP_OUT))
    x = torch.zeros((64, S.STITCH_MLP_IN), dtype=torch.int16, device="cuda")
    y = torch.empty((64, S.STITCH_MLP_OUT), dtype=torch.float32, device="cuda")
    S.stitch_mlp_forward(mlp, x, 64, y)
    assert S.stitch_mlp_status(mlp) == S.STITCH_OK
    S.stitch_mlp_inject_error(mlp, 1)
    with pytest.raises(S.StitchError) as ei:
        S.stitch_mlp_status(mlp)
    assert ei.value.code == S.STITCH_ETIMEOUT
    assert S.stitch_mlp_status(mlp) == S.STITCH_OK          # reported once, then cleared
    S.stitch_mlp_inject_error(mlp, 3)
    for _ in range(2):                                       # sticky
        with pytest.raises(S.StitchError) as ei:
            S.stitch_mlp_status(mlp)
        assert ei.value.code == S.STITCH_ETIMEOUT
    with pytest.raises(S.StitchError) as ei:
        S.stitch_mlp_forward(mlp, x, 64, y)
    assert ei.value.code == S.STITCH_ETIMEOUT
    S.stitch_mlp_set_gemm(mlp, S.STITCH_MLP_GEMM_MMA_SYNC)
    S.stitch_mlp_forward(mlp, x, 64, y)                      # the other engine still runs
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    S.stitch_mlp_destroy(mlp)
