"""CPU oracle for the low-rank NUFFT of Ruiz-Antolin and Townsend (arXiv:1701.04492).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import, call, link or execute it.  The
product library never does, and it shares no code with the CUDA path: no kernels,
headers, helpers, tables or constant generators.

Two independent references live here, both in IEEE double precision:

* ``oracle.direct``  -- the plain O(N*M) definition, eq. (1.2), written in C with an
  exact reduction of the phase x_j*k modulo 1 and compensated summation.
* ``oracle.lowrank`` -- the paper's method step by step (section 2.2 and the
  vectorised two-step form of section 2.3) in numpy, with numpy's FFT and scipy's
  Bessel function as library steps.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against values the paper prints (Table 2.1, Fig. 2.1), closed forms, brute force in
multiple precision (mpmath) and the paper's error bounds.  No function is unpinned.
"""

from . import lowrank  # noqa: F401
from . import direct  # noqa: F401
