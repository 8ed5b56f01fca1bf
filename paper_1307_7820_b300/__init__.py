"""B300-native two-vector Four-Russians Nussinov folding.

The compute path is the CUDA library ``libfold_b300.so`` (built from
``csrc/``) behind the C-ABI declared in ``include/fold.h``; :mod:`.fold` is the
thin ctypes binding with the same names.  Importing this package does not load
the library; :func:`fold.lib` does, and raises if it is missing.
"""
__all__ = ["fold", "synth"]
