"""ctypes binding of include/dirac.h (argument marshalling only).

Every computation happens in the CUDA library; if the library is missing or
cannot be loaded this module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

_lib = None

HEADER = os.path.join(_build.ROOT, "include", "dirac.h")
KRYLOV_MAX = 32
KERNEL_KINDS = 3
EIG_RITZ_MAX = 256
EIG_ITER_MAX = 8192

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ESTATE = range(6)
PERIODIC, DIRICHLET = 0, 1
FP64, MIXED = 0, 1
OBS_PX, OBS_PROJ = 0, 1
STEP_AUTO, STEP_PASSES, STEP_ONE_LAUNCH = 0, 1, 2
PEAK_FP64, PEAK_FP32 = 0, 1


class StepInfoC(ctypes.Structure):
    _fields_ = [("k_used", ctypes.c_int), ("breakdown", ctypes.c_int),
                ("err_est", ctypes.c_double), ("cum_err", ctypes.c_double),
                ("norm", ctypes.c_double), ("energy", ctypes.c_double),
                ("alpha", ctypes.c_double * KRYLOV_MAX), ("beta", ctypes.c_double * KRYLOV_MAX),
                ("kappa_max", ctypes.c_double)]


class ProblemC(ctypes.Structure):
    """dirac_problem of include/dirac.h (the allocation-free step's problem description)."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("mass", ctypes.c_double), ("c", ctypes.c_double),
                ("stencil_order", ctypes.c_int), ("boundary", ctypes.c_int),
                ("V_dev", ctypes.c_void_p), ("A_x", ctypes.c_double), ("A_y", ctypes.c_double),
                ("energy_shift", ctypes.c_double)]


class TuneResultC(ctypes.Structure):
    _fields_ = [("tile_height", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("ms_per_step", ctypes.c_double), ("from_cache", ctypes.c_int),
                ("candidates", ctypes.c_int)]


class EigInfoC(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("n_found", ctypes.c_int),
                ("n_in_window", ctypes.c_int), ("n_converged", ctypes.c_int),
                ("breakdown", ctypes.c_int), ("launches", ctypes.c_longlong),
                ("ms_apply", ctypes.c_double), ("ms_dot", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("ms_other", ctypes.c_double)]


class AdjointOptsC(ctypes.Structure):
    _fields_ = [("observable", ctypes.c_int), ("phi_dev", ctypes.c_void_p),
                ("checkpoint_every", ctypes.c_int), ("block_x", ctypes.c_int),
                ("block_y", ctypes.c_int), ("n_coef", ctypes.c_int),
                ("W_host", ctypes.POINTER(ctypes.c_double))]


class AdjointInfoC(ctypes.Structure):
    _fields_ = [("ms_forward", ctypes.c_double), ("ms_backward", ctypes.c_double),
                ("quadrature_nodes", ctypes.c_int), ("checkpoints", ctypes.c_int),
                ("launches", ctypes.c_longlong), ("ms_contract", ctypes.c_double)]


class DiracError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("dirac status %d (%s): %s" % (status, status_string(status), message))
        self.status = status


def header_functions() -> list:
    """Names of the functions declared in include/dirac.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"\b(dirac_[a-z_0-9]+)\s*\(", text)


def lib():
    """Load the built library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError("CUDA library %s not built; run paper_1407_7370_gb300.build.build()"
                           % _build.LIB)
    L = ctypes.CDLL(_build.LIB)
    vp, i, d, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    sig = {
        "dirac_create": (i, [ctypes.POINTER(vp), i, i, d, d, d, d, i, i, i, i, vp]),
        "dirac_destroy": (None, [vp]),
        "dirac_set_stream": (i, [vp, vp]),
        "dirac_set_fields": (i, [vp, vp, d, d, d]),
        "dirac_set_vector_potential": (i, [vp, d, d]),
        "dirac_lanczos_step": (i, [vp, vp, d, i, d, ctypes.POINTER(StepInfoC)]),
        "dirac_lanczos_steps": (i, [vp, vp, i, d, i, d, dp, ctypes.POINTER(StepInfoC)]),
        "dirac_propagate_host": (i, [vp, vp, i, d, i, d, dp, ctypes.POINTER(StepInfoC)]),
        "dirac_sync": (i, [vp]),
        "dirac_state_bytes": (ctypes.c_size_t, [vp]),
        "dirac_export_state": (i, [vp, vp, ctypes.c_size_t]),
        "dirac_import_state": (i, [vp, vp, ctypes.c_size_t]),
        "dirac_pulse_sin2_mean": (d, [d, d, d, d, d]),
        "dirac_pulse_sine_basis_means": (i, [i, d, i, d, dp]),
        "dirac_kernel_launches": (ctypes.c_longlong, [vp]),
        "dirac_status_string": (ctypes.c_char_p, [i]),
        "dirac_last_error": (ctypes.c_char_p, []),
        "dirac_debug_tridiag_expm": (i, [dp, dp, i, d, d, d, dp, dp]),
        "dirac_measure_peak": (i, [i, dp]),
        "dirac_profile_enable": (i, [vp, i]),
        "dirac_lanczos_step_noalloc": (i, [ctypes.POINTER(ProblemC), vp, d, i, d, vp,
                                           ctypes.POINTER(StepInfoC)]),
        "dirac_noalloc_scratch_bytes": (ctypes.c_size_t, []),
        "dirac_batch_create": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(i), ctypes.POINTER(i), dp, dp,
                                   d, d, i, i, i, i, vp]),
        "dirac_batch_destroy": (None, [vp]),
        "dirac_batch_set_fields": (i, [vp, i, vp, d, d, d]),
        "dirac_batch_set_launch_shape": (i, [vp, i, i]),
        "dirac_batch_steps": (i, [vp, ctypes.POINTER(vp), i, d, i, d, dp, ctypes.POINTER(StepInfoC)]),
        "dirac_batch_sync": (i, [vp, ctypes.POINTER(StepInfoC)]),
        "dirac_batch_profile_enable": (i, [vp, i]),
        "dirac_batch_profile_read": (i, [vp, dp, ctypes.POINTER(ctypes.c_longlong)]),
        "dirac_batch_kernel_launches": (ctypes.c_longlong, [vp]),
        "dirac_batch_autotune": (i, [vp, ctypes.POINTER(vp), d, i, dp, i, ctypes.POINTER(TuneResultC)]),
        "dirac_batch_use_graphs": (i, [vp, i]),
        "dirac_use_graphs": (i, [vp, i]),
        "dirac_set_step_mode": (i, [vp, i]),
        "dirac_batch_set_step_mode": (i, [vp, i]),
        "dirac_debug_barrier_timeout": (i, [vp, vp, d, i]),
        "dirac_profile_read": (i, [vp, dp, ctypes.POINTER(ctypes.c_longlong)]),
        "dirac_apply_hamiltonian": (i, [vp, vp, vp]),
        "dirac_lanczos_eigs": (i, [vp, vp, i, i, i, d, d, d, i, i, d, dp, dp, vp,
                                   ctypes.POINTER(EigInfoC)]),
        "dirac_adjoint_gradient": (i, [vp, vp, i, d, i, dp, ctypes.POINTER(AdjointOptsC), dp, vp, vp,
                                       dp, dp, ctypes.POINTER(AdjointInfoC)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(s: int) -> str:
    try:
        return lib().dirac_status_string(s).decode()
    except Exception:  # pragma: no cover - only used in error paths
        return "?"


def check(status: int) -> None:
    if status != OK:
        raise DiracError(status, lib().dirac_last_error().decode())
