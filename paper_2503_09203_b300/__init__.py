"""B300-native batched UUV step of MarineGym (arXiv 2503.09203).

The compute path is the CUDA library ``libmarinegym.so`` behind the C-ABI in
``include/marinegym.h``; :mod:`paper_2503_09203_b300.binding` is its thin
ctypes binding. Importing this package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
__all__ = ["binding", "vehicles", "workloads"]
