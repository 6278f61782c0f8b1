"""GB300-native demag + LLG hot path of a finite-difference micromagnetic
solver (Zhu, "Speedup of Micromagnetic Simulations with C++ AMP on GPUs").

The compute runs in the hand-written sm_103a kernels of ``libmm.so`` behind a
C ABI (``include/mm.h``); ``paper_1406_7459_gb300.mm`` is the thin ctypes
binding with the same names.  Importing this package does not load the
library; the first binding call does, and raises if it is missing.
"""
