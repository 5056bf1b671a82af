"""GB300 (sm_103a) ST-HOSVD Tucker compression: CUDA kernels behind a C ABI.

``tucker`` is the ctypes binding of ``include/tucker.h``; ``build`` compiles
the library in-tree with nvcc.
"""
__all__ = ["tucker", "build"]
