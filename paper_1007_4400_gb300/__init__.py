"""GB300-native solver for sequences of dense complex Hermitian-definite generalized
eigenproblems A x = lambda B x (warm-started Chebyshev-filtered subspace iteration).

The compute path is libgevp (hand-written CUDA for sm_103a behind the C ABI in
include/gevp.h); this package holds the ctypes binding and the seeded input generator.
"""
from . import synth  # noqa: F401
from . import gevp  # noqa: F401

__all__ = ["synth", "gevp"]
