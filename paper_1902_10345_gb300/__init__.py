"""GB300-native iterated Jacobi-2D stencil library (sm_103a CUDA kernels behind a C ABI).

The compute path lives in ``csrc/`` and is reached through ``binding`` (a thin
ctypes layer over ``libsdfgjacobi.so``).  Importing this package does not load
the shared library; ``binding.lib()`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "binding"]
