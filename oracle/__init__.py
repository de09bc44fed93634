"""FP64 CPU oracle of the ROK hot path (Sec. 2.2.2, Eq. ROK; Sec. 2.3, Eq. matvecFD;
Sec. 3.2, Eq. Nav_Stokes).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never
imports, links or calls anything in this package, and this package never
imports the product library.  It is plain, slow code (single-threaded; the
OpenMP build of ``residual.c`` that times the CPU baseline on every host core
computes the same bits):
the residual and the finite-difference JVP in C (``residual.c``, compiled
with ``-ffp-contract=off``), the time integrators in NumPy
(``integrators.py``), the coefficient tables in ``coefficients.py``.
"""
