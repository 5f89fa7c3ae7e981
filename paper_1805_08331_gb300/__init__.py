"""GB300-native entropic optimal transport between persistence diagrams.

The compute path is a C-ABI CUDA library (``csrc/``, declared in
``include/pd_ot.h``) built for sm_103a; ``api`` is a thin ctypes binding with
the same names.  Importing this package does not load the library; the first
call through ``api`` does, and fails loudly if it is missing.
"""
__all__ = ["api", "inputs"]
