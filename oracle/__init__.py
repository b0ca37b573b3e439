"""Plain FP64 CPU oracle for the second-generation spherical curvelet transform
(Chan, Leistedt, Kitching, McEwen, arXiv:1511.05578).

TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the CPU-baseline leg of
the benchmark may import this package. The product library never imports, links or
runs it, and it shares no code, table or helper with the CUDA path: the two meet
only at the seeded input generator, which holds none of the method's arithmetic.

Layout:
  orc.c        C inner loops (Wigner d by two methods, Risbo Delta, O(L^4) sums)
  curvelet.py  numpy layer: sampling grids, spin SHT, kernels, analysis, synthesis
  build.py     gcc build of orc.c

Parity status of each function is stated in its docstring; every function here is
pinned by a test in tests/test_oracle_*.py against something other than itself
(the paper's closed forms, the factorial sum, brute force at tiny L, scipy, exact
reconstruction, admissibility).
"""
from .curvelet import *  # noqa: F401,F403
