"""GB300-native (sm_103a) single-pulse search hot path of ASTROFLOW
(arXiv 2511.02328): brute-force dedispersion, boxcar S/N and candidates.

The compute lives in libafgb.so (C ABI in include/afgb.h); `_lib` is its
ctypes binding, `search.Plan` a torch-facing helper, `synth` the seeded
input generator.
"""
from . import _lib  # noqa: F401

__all__ = ["_lib"]
