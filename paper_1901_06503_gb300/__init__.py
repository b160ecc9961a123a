"""GB300-native one-step full-field photoacoustic reconstruction.

The compute path is the CUDA library ``libffpat.so`` behind the C ABI in
``include/ffpat.h``; :mod:`paper_1901_06503_gb300.ffpat` is its thin ctypes
binding.  Importing this package loads nothing; the library is loaded on the
first call of the binding and a missing library is an error (there is no CPU
fallback).
"""
__all__ = ["ffpat", "inputs"]
