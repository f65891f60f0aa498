"""CPU FP64 oracle for the Dirac Lanczos propagator -- TEST INFRASTRUCTURE ONLY.

A plain, slow, readable restatement of what the paper computes, used to check
the CUDA path.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library itself
never does, and this package imports nothing from the library (it shares only
the seeded input generators of ``paper_1407_7370_gb300.workloads``, which hold
none of the method's arithmetic).

Modules
-------
hamiltonian  the discretised 2D two-component Dirac operator (Sec. 3, Eq. 12)
lanczos      Fig. 1 recurrence (MGS form, Eq. 4), Krylov exponential step
             (Eq. 17), its error estimate (Eq. 18), and the eigenvalue mode with
             full reorthogonalisation (Sec. 2, Eqs. 9-10; Sec. 5)
free         closed-form propagator of the free discretised operator (uniform
             vector potential): exact per Fourier mode, for pinning the above
fields       first-order Magnus field average over a step (Eq. 16)

Every function here has a pin in ``tests/test_oracle_*.py`` against something
other than itself (closed forms, library routines, invariants).
"""
from . import hamiltonian, lanczos, free, fields  # noqa: F401
