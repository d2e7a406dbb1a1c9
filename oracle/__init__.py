"""The oracle: a plain, slow, FP64 CPU implementation of the multi-level
constrained-realization solver's hot path (Seljebotn et al. 2013,
arXiv:1308.5299).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in
this package.  The product library (``paper_1308_5299_gb300``) never imports
it and shares no code with it; the two meet only through the seeded input
generators in ``paper_1308_5299_gb300/synthetic.py``, which hold none of the
method's arithmetic.

Modules
  geometry    HEALPix and Gauss-Legendre ring grids (Section 2.1)
  sht         direct FP64 synthesis Y / adjoint Y^T (Eq. sh-synthesis), C core
  operators   S, B, N^-1, A and the level operators A_h (Eqs. system-explicit, A_h)
  solvers     dense Cholesky solve, diagonal-preconditioned CG (Section 2.4)
  multilevel  filters, restriction, pixel smoother, CR-Cycle / CR-Solve
              (Sections 3.2-3.5, Fig. code:mg)
  rng         Philox4x32-10 + Box-Muller, from the published definitions
"""
