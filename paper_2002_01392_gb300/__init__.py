"""GB300 (sm_103a) FC-Gram pseudospectral Navier-Stokes hot path.

The compute lives in ``libfcns.so`` (hand-written CUDA kernels behind a C ABI
declared in ``include/fcns.h``).  ``paper_2002_01392_gb300.api`` is a thin
ctypes binding with the same names; it only marshals arguments.  Importing
this package does not load the library; ``api`` does, and raises if it is
missing (there is no CPU fallback).
"""

__all__ = ["api", "build"]
