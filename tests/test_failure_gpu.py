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
