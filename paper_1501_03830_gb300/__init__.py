"""GB300-native structure-preserving Bethe--Salpeter eigensolver.

The solver lives in a C-ABI shared library (``libbse_gb300.so``, built from
``csrc/`` for sm_103a); :mod:`paper_1501_03830_gb300.bse` is a thin ctypes
binding with the same entry-point names. Importing this package does not load
the library; ``from paper_1501_03830_gb300 import bse`` does, and fails loudly
if it has not been built.
"""
