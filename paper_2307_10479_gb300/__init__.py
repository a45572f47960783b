"""GB300-native batched search over a Dynamic Exploration Graph (DEG, arXiv 2307.10479).

The compute path lives in ``libdeg.so`` (hand-written CUDA for sm_103a behind a C ABI declared
in ``include/deg.h``); this package is a thin ctypes binding with the same names. Importing the
package does not load the library; the first call does, and raises if it is missing.
"""
