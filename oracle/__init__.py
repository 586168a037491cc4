"""FP64 CPU oracle for the DiffBMP rasterizer -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA library and the library never
calls it.  See ``dbmp_oracle.c`` for the equations it follows.
"""
from .oracle import *  # noqa: F401,F403
