"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This package only draws inputs (anchor sets, decoder weights, cameras, trajectories,
random Gaussians/records/keys for stage tests).  It contains none of the renderer's
arithmetic (selection, decoding, projection, sorting, blending); both the FP64 oracle
and the CUDA path consume what it produces.
"""
from .scenes import *  # noqa: F401,F403
