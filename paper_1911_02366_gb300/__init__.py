"""GB300 (sm_103a) statically condensed GL-DGSEM Newton solver.

The compute path is the CUDA library ``_build/libsc.so`` (C ABI in include/sc.h);
``paper_1911_02366_gb300.sc`` is a thin ctypes binding with the same names.
Importing this package does not load the library; ``sc.lib()`` does, and raises if
the library is missing (there is no CPU fallback).
"""
__all__ = ["sc", "build"]
