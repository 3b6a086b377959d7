"""GB300-native Q1 matrix-free finite-element operators and Krylov solvers.

The compute path is the C-ABI library ``libmf.so`` built from ``csrc/`` (CUDA for sm_103a); the
Python module ``mf`` is a thin ctypes binding to it.  Importing this package does not load the
library; ``paper_2308_09839_gb300.mf`` does, and raises if it has not been built.
"""
