"""CPU FP64 oracle for the multiscreen hypersingular BEM hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product library (``paper_2310_09204_gb300``) never imports
it, and it never imports the product library (it shares only the seeded input
generators of ``paper_2310_09204_gb300.workloads``, which hold no arithmetic
of the method).

Layout:
  oracle_core.c  quadrature rules and the dense single-layer pair matrix V (C)
  core.py        ctypes binding / build of oracle_core.c
  topology.py    sectors, generalized vertices, dofs, curl lists, patch
                 classes and coarse prolongation (Sec. 4.2-4.3, Sec. 5)
  solver.py      W = sum_k S_k^T V S_k, RHS, additive Schwarz preconditioner,
                 PCG and the Lanczos condition-number estimate (Sec. 2.1)
"""
