"""GB300-native sampler for gauged superpositions of Gaussian fermionic PEPS.

The compute path is libggf.so (hand-written CUDA for sm_103a behind a C ABI,
include/ggf.h); this package only builds it and marshals arguments.  There is
no CPU fallback: importing the binding fails loudly when the library is
missing.
"""
from .ggf import GGF, GGFError, Net, Z2, U1, SU2, FP64, FP32, lib_path, sample_group  # noqa: F401
