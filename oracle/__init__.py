"""Plain FP64 CPU oracle of the video-stitching hot path (arXiv 2308.09209).

TEST INFRASTRUCTURE ONLY. This package exists to check the CUDA path: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import, call or execute anything in it. The product path
(the C-ABI library and its Python binding) never imports it and has no CPU
fallback. The oracle shares no code with the CUDA path: no kernels, headers,
helpers, tables or pre/post-processing. Both sides only consume the same
seeded inputs from the separate ``synth`` package.

Every function follows the paper's definitions in the order the paper gives
them, in float64 (integer statistics in int64), with no blocking, fusion or
reordering beyond what the definition states. Modules:

* ``geometry``  -- overlap determination (section 2.1 step 1; section 3.1):
  homography inverse, coverage, overlap bands, source rectangles, colour
  pair directions toward the reference camera.
* ``color``     -- 3D-M colour transfer (section 2.1 steps 2-5, Eq. 1-4):
  histograms, histogram specification, normal equations over the temporal
  window, the 3x3 solve, chaining to the reference camera.
* ``balance``   -- online colour balancing (section 2.2, Eq. 5-7): lambda
  quantile knots, 3-frame knot smoothing, the piecewise gamma/linear/gamma
  curve.
* ``warp``      -- pre-warp, optical-flow local warping and weighted-mean
  fusion (section 3.1, section 3.2, Eq. 15-18), per pixel.
* ``pipeline``  -- the per-frame sequence with its temporal state.
* ``refine``    -- homography refinement from the band flows (section 3.1,
  Eq. 13-14, with the supplied flow fields in place of SURF matches).
* ``flow``      -- optical flow between a pair's pre-warped images over its
  blend band (section 3.2), a coarse-to-fine integer block matcher.
* ``correspondence`` -- the one-frame colour transfer from pixel
  correspondences that Tables 2-3 compare against (2D-M).

Parity pins: each function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or a library routine (see each test
module). Parts that are readings of the paper rather than the paper's own
definition (the balance targets d1/d2, the flow-weight swap in Eq. 17, the
pooled balance histogram, the chained M) are pinned for internal consistency
only: parity against the paper's own results is unpinned for those readings,
because the paper prints no worked example for them.
"""
from . import geometry, color, balance, warp, pipeline  # noqa: F401
from .pipeline import OracleStitcher  # noqa: F401

BALANCE_OFF = 1
FP16_INTERMEDIATE = 2
FLOW_WEIGHTS_PRINTED = 4
LEARNED = 8
BALANCE_OUTPUT = 16
