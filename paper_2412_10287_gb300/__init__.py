"""GB300-native single-source 2-RPQ (arXiv:2412.10287).

The compute path lives in the CUDA library ``librpq.so`` behind the C ABI of
``include/rpq.h``; :mod:`paper_2412_10287_gb300.rpq` is its ctypes binding.
Importing this package loads nothing: the binding loads the library on first
use and raises if it is missing.
"""
