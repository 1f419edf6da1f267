"""CPU FP64 oracle for the Newton-step Krylov solve of arXiv 1709.05660.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the ``libfsi`` C-ABI library and its Python
binding) never calls it; the two share no code besides the seeded input
generators of ``paper_1709_05660_gb300.workloads``.

The oracle is plain and slow on purpose: numpy / scipy in float64, each step
written in the paper's order with a citation of the section or equation it
follows.  Modules:

* ``mesh``   - mesh hierarchy, unknown numbering, node classes, Dirichlet data,
               Schwarz patches (Sec. 2.5, 3.1, 3.2, 3.3).
* ``fem``    - Q2-P1disc residual of the steady (and BDF2) monolithic weak form
               and its exact Jacobian by forward-mode dual numbers (Sec. 2.3,
               2.5, 3).
* ``solver`` - prolongation / restriction, Galerkin coarse operators,
               Richardson-Schwarz smoother, V-cycle, FGMRES, the direct
               solve and the Newton driver (Sec. 3, 3.2, 3.3, 4.1).

Parity pins: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, a brute-force or library computation, or the
paper's printed integers (see ``tests/test_oracle_*.py``).
"""
