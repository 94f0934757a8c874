"""GB300-native BVH traversal with subspace culling (Yoshimura & Harada, 2023).

The product is ``libsubcull.so`` (C-ABI declared in include/subcull.h); the
Python modules here only marshal arguments:
  - ``subcull``   : ctypes binding with the C-ABI's names (sc_*),
  - ``scenegen``  : seeded synthetic inputs (shared with the CPU oracle).
"""
__all__ = ["subcull", "scenegen"]
