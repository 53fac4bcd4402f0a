"""B300-native video-stitching hot path (arXiv 2308.09209) behind a C ABI.

``stitch`` is the ctypes binding of libstitch.so (include/stitch.h); ``build``
compiles the library in-tree for sm_103a.
"""
from . import stitch  # noqa: F401
from .stitch import Config, Stitcher, StitchError  # noqa: F401
