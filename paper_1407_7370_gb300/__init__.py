"""GB300-native Dirac Lanczos propagator (Beerwerth & Bauke, arXiv:1407.7370).

``Propagator`` advances a two-component spinor on a uniform 2D grid by the
Krylov (Lanczos) approximation of exp(-i H dt) with H the finite-difference
Dirac Hamiltonian (Sec. 3-4 and 7 of the paper).  All work runs in the CUDA
library behind ``include/dirac.h``; PyTorch tensors only provide device memory
and the stream.
"""
from .propagator import (BatchPropagator, EigResult, Propagator, StepInfo, pulse_sin2_mean,  # noqa: F401
                         tridiag_expm_device)
from . import workloads  # noqa: F401
