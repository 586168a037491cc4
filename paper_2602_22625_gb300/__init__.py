"""GB300 (sm_103a) differentiable rasterizer for bitmap primitives (DiffBMP).

The compute path is libdbmp.so (CUDA, built in-tree by ``_build.build()``) behind the
C ABI of ``include/dbmp.h``; ``dbmp`` is its ctypes binding, ``render`` the renderer
objects and autograd wrapper, ``inputs`` the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
