"""GB300-native (sm_103a) NeuralPVS hot path: froxelization, 3-D interleave, sparse convolution
network and de-interleave behind the npvs C ABI (include/npvs.h, libnpvs.so).

Importing the package is light; the CUDA library is loaded on first use and its absence is an
error (there is no fallback implementation).
"""
from . import _lib  # noqa: F401

__all__ = ["ops", "pipeline"]
