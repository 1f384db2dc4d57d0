"""libmpjacobi: a GB300-native mixed precision Jacobi eigensolver.

The compute path is the C-ABI shared library ``libmpjacobi.so`` built from
``csrc/`` (CUDA for sm_103a); ``mpj`` is a thin ctypes binding with the same
entry-point names.  Importing this package loads nothing: the library is loaded
by the first call into ``mpj``, which raises if it is missing.
"""
__all__ = ["mpj", "inputs"]
