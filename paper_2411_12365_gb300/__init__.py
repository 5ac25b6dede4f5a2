"""GB300-native Bumped Ribbon Retrieval (BuRR) construction and query.

The compute path lives in ``libburr.so`` (hand-written sm_103a CUDA behind a
C ABI declared in ``include/burr.h``); ``burr`` is the thin ctypes binding.
Importing the package does not load the library; the first call does, and it
raises if the library is missing.
"""
__all__ = ["burr", "inputs"]
