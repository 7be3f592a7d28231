"""CPU oracle for the SSAMG hot path (test infrastructure only).

A plain, slow, FP64 numpy restatement of the semi-structured algebraic
multigrid method of Magri, Falgout and Yang (arXiv 2205.14273), written from
the paper's text: coarsening (Section 3.1, Algorithm 1), operator-based
two-point interpolation (Section 3.2, Eq. prolEx), Galerkin coarse operators
(Section 3.3, Eq. galerkin), weighted / L1 Jacobi relaxation (Section 3.4,
Eqs. relax0, relax1, alpha-beta), the V(1,1) cycle and preconditioned CG
(Section 4).  ``assembled`` is an independent brute-force checker built on
scipy CSR matrices.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
shares no code with the library: the two meet only in the seeded input
generators of the ``problems`` package.
"""
from .ssamg import *  # noqa: F401,F403
