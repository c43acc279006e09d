"""GB300 (sm_103a) Hermite block-timestep direct N-body library.

The compute path is libnbody.so (CUDA, C ABI in include/nbody.h); this package
holds its sources (csrc/), the in-tree build (``build()``) and the ctypes
binding (``nbody``).
"""
from ._build import build, LIB as LIB_PATH  # noqa: F401
from . import nbody  # noqa: F401
