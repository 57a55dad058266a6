"""GB300 (sm_103a) RHEED/TRHEPD rocking-curve engine: the matrix-ODE multi-slice method with the
right-hand-side transformation (Kudo, Yamamoto & Hoshi), behind the C-ABI library ``libtrheed``.

Importing the package loads nothing native; ``paper_2306_00271_gb300.api`` loads the library and
raises if it is missing (there is no CPU fallback).
"""
__all__ = ["workloads"]
