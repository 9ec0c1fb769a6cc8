"""GB300-native matching pursuit on multi-Gabor dictionaries.

Prusa, Holighaus, Balazs, "Fast Matching Pursuit with Multi-Gabor
Dictionaries" (ACM TOMS 47(3), 2021): coefficient-domain MP with truncated,
precomputed cross-Gram kernels.  The compute path is the CUDA library
libmpgabor.so (C ABI in include/mpgabor.h); ``mpgabor`` is its Python
binding, ``inputs`` the seeded synthetic inputs, ``build`` the nvcc build.

Importing this package does not load the CUDA library; ``mpgabor.lib()``
does, and fails loudly if it has not been built.
"""
__all__ = ["mpgabor", "inputs", "build"]
