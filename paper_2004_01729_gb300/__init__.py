"""GB300-native finite-temperature CCSD (White & Chan, arXiv:2004.01729).

The compute path lives in the CUDA/C++ library ``libftcc`` (``csrc/``),
exposed through the C ABI declared in ``include/ftcc.h``; ``ftcc.py`` is the
thin ctypes binding with the same entry-point names.  Importing this package
does not load the library; ``ftcc.load()`` does, and raises if it is missing.
"""
