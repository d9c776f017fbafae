"""GB300-native extended-stencil FDTD (Blinne et al., arXiv:1710.06829).

The compute path is libfdtd.so (hand-written CUDA for sm_103a behind the C ABI
of include/fdtd.h).  ``_lib`` is the ctypes binding with the C entry-point
names; ``sim`` wraps a handle with torch tensors for device memory; ``inputs``
holds the seeded synthetic input generators.
"""
from . import _lib  # noqa: F401

__all__ = ["_lib", "sim", "inputs"]
