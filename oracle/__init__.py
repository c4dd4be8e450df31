"""CPU FP64 oracle for the MASW theoretical dispersion curve.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, the package smoke check and the
benchmark's CPU-baseline leg. It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
