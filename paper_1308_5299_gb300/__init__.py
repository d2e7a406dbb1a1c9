"""GB300-native multi-level constrained-realization solver (Seljebotn et al.
2013, arXiv:1308.5299): the spherical-harmonic-transform-based application of
A = S^-1 + B Y^T N^-1 Y B inside the multi-level W-cycle, as hand-written
CUDA kernels for sm_103a behind a C ABI (``include/cr.h``).

``paper_1308_5299_gb300.binding`` is the thin ctypes binding over the shared
library; it loads the library on first use and raises if it is missing (there
is no CPU fallback).  ``paper_1308_5299_gb300.synthetic`` generates seeded
input data.
"""
