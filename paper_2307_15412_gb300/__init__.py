"""GB300-native radar ray-tracing hot path (arXiv 2307.15412).

Submodules:
  inputs -- seeded synthetic scenes, radar and ray-grid descriptions
  rr     -- ctypes binding of the C ABI (include/rr.h) over librr.so
  build  -- in-tree nvcc build of librr.so for sm_103a
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "rr", "build"]
