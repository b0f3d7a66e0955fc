"""GB300-native weighted NMF for coronagraphic PSF subtraction (arXiv:2309.04623).

The compute path is libnmfgb.so (hand-written CUDA for sm_103a behind a C-ABI,
include/nmf.h); `nmf` is its Python binding and `synthetic` the seeded
generator of the reference libraries and science frames.
"""
from . import synthetic  # noqa: F401

__all__ = ["synthetic", "nmf", "build"]
