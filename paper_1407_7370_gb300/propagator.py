"""Python front end of the C ABI: a thin object over dirac_create/.../dirac_destroy."""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _native as nat


@dataclasses.dataclass
class StepInfo:
    k_used: int
    breakdown: bool
    err_est: float
    cum_err: float
    norm: float
    energy: float
    alpha: np.ndarray
    beta: np.ndarray
    kappa_max: float = 0.0


def _info(c: nat.StepInfoC) -> StepInfo:
    k = c.k_used
    return StepInfo(k, bool(c.breakdown), c.err_est, c.cum_err, c.norm, c.energy,
                    np.array(c.alpha[:k]), np.array(c.beta[:k]), c.kappa_max)


@dataclasses.dataclass
class EigResult:
    """Result of Propagator.eigs (energies of H - shift)."""
    values: np.ndarray       # ascending
    bounds: np.ndarray       # Eq. 9 bounds (folded mode: bounds on lambda)
    iterations: int
    n_in_window: int
    n_converged: int
    breakdown: bool
    vectors: object = None   # CUDA complex128 tensor (n, ny, nx, 2) of unit Ritz vectors, or None
    launches: int = 0
    ms: dict = None          # device ms per kernel kind while profiling (apply, dot, update, other)


@dataclasses.dataclass
class AdjointResult:
    """Result of Propagator.adjoint_gradient."""
    loss: float
    dV: object = None        # CUDA float64 tensor (ny / by, nx / bx): dL/dV summed over blocks
    dA: np.ndarray = None    # (nsteps, 2): dL/dA_x, dL/dA_y of every step
    da: np.ndarray = None    # (n_coef,): dL/da_k for A_x = W a
    psiN: object = None      # CUDA complex128 tensor (ny, nx, 2): the final state
    info: dict = None


def _torch():
    import torch
    return torch


def _stream_ptr():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check_psi(psi, ny, nx):
    torch = _torch()
    if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
        raise TypeError("psi must be a CUDA torch tensor")
    if psi.dtype != torch.complex128 or tuple(psi.shape) != (ny, nx, 2) or not psi.is_contiguous():
        raise ValueError("psi must be contiguous complex128 of shape (%d, %d, 2)" % (ny, nx))


class Propagator:
    """Lanczos propagator for one grid; see include/dirac.h for the semantics."""

    def __init__(self, nx: int, ny: int, dx: float, dy: float, mass: float = 1.0,
                 c: float = 137.036, order: int = 2, boundary: str = "periodic", m_max: int = 20,
                 precision: str = "fp64"):
        L = nat.lib()
        self.nx, self.ny = nx, ny
        b = {"periodic": nat.PERIODIC, "dirichlet": nat.DIRICHLET}[boundary]
        prec = {"fp64": nat.FP64, "mixed": nat.MIXED}[precision]
        self._ctx = ctypes.c_void_p()
        self._stream = _stream_ptr()
        nat.check(L.dirac_create(ctypes.byref(self._ctx), nx, ny, dx, dy, mass, c, order, b,
                                 prec, m_max, self._stream))

    def _sync_stream(self):
        s = _stream_ptr()
        if s.value != self._stream.value:
            nat.check(nat.lib().dirac_set_stream(self._ctx, s))
            self._stream = s

    def set_fields(self, V=None, A=(0.0, 0.0), shift: float = 0.0):
        """V: CUDA float64 tensor (ny, nx) of potential energy, or None."""
        self._sync_stream()
        ptr = None
        if V is not None:
            torch = _torch()
            if V.dtype != torch.float64 or not V.is_cuda or tuple(V.shape) != (self.ny, self.nx) \
                    or not V.is_contiguous():
                raise ValueError("V must be a contiguous CUDA float64 tensor (ny, nx)")
            ptr = ctypes.c_void_p(V.data_ptr())
        nat.check(nat.lib().dirac_set_fields(self._ctx, ptr, float(A[0]), float(A[1]), float(shift)))

    def set_vector_potential(self, ax: float, ay: float = 0.0):
        nat.check(nat.lib().dirac_set_vector_potential(self._ctx, float(ax), float(ay)))

    def step(self, psi, dt: float, m: int, tol: float = 0.0, info: bool = False):
        return self.steps(psi, 1, dt, m, tol, None, info)

    def steps(self, psi, nsteps: int, dt: float, m: int, tol: float = 0.0, A=None,
              info: bool = False):
        """nsteps in place; A: optional (nsteps, 2) array of per-step vector potentials."""
        _check_psi(psi, self.ny, self.nx)
        self._sync_stream()
        a_ptr, a_arr = None, None
        if A is not None:
            a_arr = np.ascontiguousarray(A, dtype=np.float64).reshape(nsteps, 2)
            a_ptr = a_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        out = nat.StepInfoC() if info else None
        nat.check(nat.lib().dirac_lanczos_steps(self._ctx, ctypes.c_void_p(psi.data_ptr()), nsteps,
                                                dt, m, tol, a_ptr,
                                                ctypes.byref(out) if info else None))
        return _info(out) if info else None

    def propagate_host(self, psi_host, nsteps: int, dt: float, m: int, tol: float = 0.0, A=None):
        """psi_host: host complex128 (ny, nx, 2) buffer (numpy array or pinned CPU tensor),
        updated in place; host<->device copies happen inside the call."""
        if isinstance(psi_host, np.ndarray):
            if psi_host.dtype != np.complex128 or psi_host.shape != (self.ny, self.nx, 2) \
                    or not psi_host.flags.c_contiguous:
                raise ValueError("psi_host must be C-contiguous complex128 (ny, nx, 2)")
            ptr = psi_host.ctypes.data
        else:
            torch = _torch()
            if psi_host.is_cuda or psi_host.dtype != torch.complex128 or not psi_host.is_contiguous():
                raise ValueError("psi_host must be a contiguous CPU complex128 tensor")
            ptr = psi_host.data_ptr()
        self._sync_stream()
        a_ptr, a_arr = None, None
        if A is not None:
            a_arr = np.ascontiguousarray(A, dtype=np.float64).reshape(nsteps, 2)
            a_ptr = a_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        out = nat.StepInfoC()
        nat.check(nat.lib().dirac_propagate_host(self._ctx, ctypes.c_void_p(ptr), nsteps, dt, m,
                                                 tol, a_ptr, ctypes.byref(out)))
        return _info(out)

    def sync(self):
        nat.check(nat.lib().dirac_sync(self._ctx))

    def apply(self, psi, out=None):
        """out = (H - shift) psi on the device (FP64); returns out."""
        _check_psi(psi, self.ny, self.nx)
        if out is None:
            out = _torch().empty_like(psi)
        _check_psi(out, self.ny, self.nx)
        self._sync_stream()
        nat.check(nat.lib().dirac_apply_hamiltonian(self._ctx, ctypes.c_void_p(psi.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr())))
        return out

    def eigs(self, start, n_want: int, max_iter: int, tol: float, window=None,
             check_every: int = 10, reorth: bool = True, fold=None, vectors: bool = False) -> EigResult:
        """Eigenvalue mode (dirac_lanczos_eigs): Ritz values of H - shift in ``window``
        (direct) or nearest ``fold`` (Lanczos on (H - shift - fold)^2)."""
        _check_psi(start, self.ny, self.nx)
        self._sync_stream()
        lo, hi = (window if window is not None else (0.0, 0.0))
        vals = (ctypes.c_double * n_want)()
        bnds = (ctypes.c_double * n_want)()
        vec_t = None
        if vectors:
            vec_t = _torch().empty((n_want, self.ny, self.nx, 2), dtype=start.dtype, device=start.device)
        info = nat.EigInfoC()
        nat.check(nat.lib().dirac_lanczos_eigs(
            self._ctx, ctypes.c_void_p(start.data_ptr()), n_want, max_iter, check_every, float(tol),
            float(lo), float(hi), 1 if reorth else 0, 0 if fold is None else 1,
            0.0 if fold is None else float(fold), vals, bnds,
            ctypes.c_void_p(vec_t.data_ptr()) if vec_t is not None else None, ctypes.byref(info)))
        nf = info.n_found
        return EigResult(np.array(vals[:nf]), np.array(bnds[:nf]), info.iterations,
                         info.n_in_window, info.n_converged, bool(info.breakdown),
                         vec_t[:nf] if vec_t is not None else None, int(info.launches),
                         {"apply": info.ms_apply, "dot": info.ms_dot, "update": info.ms_update,
                          "other": info.ms_other})

    def adjoint_gradient(self, psi0, nsteps: int, dt: float, m: int, A, observable: str = "px",
                         phi=None, checkpoint_every: int = 50, block=(1, 1), W=None,
                         grad_V: bool = True, grad_A: bool = True, return_state: bool = False
                         ) -> AdjointResult:
        """dirac_adjoint_gradient: L of psi_N and its gradients with respect to V
        (summed over blocks (by, bx)) and the per-step vector potential A
        ((nsteps, 2) array of step means); with W (nsteps x K), also dL/da for
        A_x = W a."""
        torch = _torch()
        _check_psi(psi0, self.ny, self.nx)
        self._sync_stream()
        A = np.ascontiguousarray(A, dtype=np.float64).reshape(nsteps, 2)
        opts = nat.AdjointOptsC()
        opts.observable = {"px": nat.OBS_PX, "proj": nat.OBS_PROJ}[observable]
        if phi is not None:
            _check_psi(phi, self.ny, self.nx)
            opts.phi_dev = phi.data_ptr()
        opts.checkpoint_every = int(checkpoint_every)
        by, bx = int(block[0]), int(block[1])
        opts.block_x, opts.block_y = bx, by
        W_arr = None
        if W is not None:
            W_arr = np.ascontiguousarray(W, dtype=np.float64).reshape(nsteps, -1)
            opts.n_coef = W_arr.shape[1]
            opts.W_host = W_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        loss = ctypes.c_double()
        dV = torch.empty((self.ny // by, self.nx // bx), dtype=torch.float64,
                         device=psi0.device) if grad_V else None
        dA = np.zeros((nsteps, 2)) if grad_A else None
        da = np.zeros(opts.n_coef) if (grad_A and W_arr is not None) else None
        psiN = torch.empty_like(psi0) if return_state else None
        info = nat.AdjointInfoC()
        dptr = ctypes.POINTER(ctypes.c_double)
        nat.check(nat.lib().dirac_adjoint_gradient(
            self._ctx, ctypes.c_void_p(psi0.data_ptr()), nsteps, dt, m,
            A.ctypes.data_as(dptr), ctypes.byref(opts), ctypes.byref(loss),
            ctypes.c_void_p(psiN.data_ptr()) if psiN is not None else None,
            ctypes.c_void_p(dV.data_ptr()) if dV is not None else None,
            dA.ctypes.data_as(dptr) if dA is not None else None,
            da.ctypes.data_as(dptr) if da is not None else None, ctypes.byref(info)))
        return AdjointResult(loss.value, dV, dA, da, psiN,
                             {"ms_forward": info.ms_forward, "ms_backward": info.ms_backward,
                              "quadrature_nodes": info.quadrature_nodes,
                              "checkpoints": info.checkpoints, "launches": int(info.launches),
                              "ms_contract": info.ms_contract})

    def use_graphs(self, enable: bool = True):
        nat.check(nat.lib().dirac_use_graphs(self._ctx, 1 if enable else 0))

    def export_state(self) -> bytes:
        """The device scalars carried between steps (see dirac_export_state):
        with psi, a checkpoint from which import_state resumes bitwise."""
        L = nat.lib()
        n = L.dirac_state_bytes(self._ctx)
        buf = ctypes.create_string_buffer(n)
        nat.check(L.dirac_export_state(self._ctx, buf, n))
        return buf.raw

    def import_state(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        nat.check(nat.lib().dirac_import_state(self._ctx, buf, len(state)))

    def set_step_mode(self, mode: str = "auto"):
        """'auto', 'passes' or 'one_launch' (see dirac_set_step_mode)."""
        code = {"auto": nat.STEP_AUTO, "passes": nat.STEP_PASSES, "one_launch": nat.STEP_ONE_LAUNCH}[mode]
        nat.check(nat.lib().dirac_set_step_mode(self._ctx, code))

    def profile(self, enable: bool = True):
        """Start/stop per-kernel CUDA-event timing (see dirac_profile_enable)."""
        nat.check(nat.lib().dirac_profile_enable(self._ctx, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kind: (total ms, launches)} since the previous read; kinds 'pass',
        'recombine' and 'step' (the one-launch step, see set_step_mode)."""
        ms = (ctypes.c_double * nat.KERNEL_KINDS)()
        n = (ctypes.c_longlong * nat.KERNEL_KINDS)()
        nat.check(nat.lib().dirac_profile_read(self._ctx, ms, n))
        return {"pass": (ms[0], n[0]), "recombine": (ms[1], n[1]), "step": (ms[2], n[2])}

    @property
    def kernel_launches(self) -> int:
        return int(nat.lib().dirac_kernel_launches(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            nat.lib().dirac_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pulse_sin2_mean(t0: float, dt: float, a0: float, omega: float, duration: float) -> float:
    """Magnus-1 mean of A0 sin^2(pi t/T) sin(omega t) over [t0, t0+dt] (library, closed form)."""
    return float(nat.lib().dirac_pulse_sin2_mean(t0, dt, a0, omega, duration))


def pulse_schedule(t0: float, dt: float, nsteps: int, a0: float, omega: float, duration: float):
    """(nsteps, 2) per-step vector potentials (A_x mean, 0) for a sin^2 pulse."""
    out = np.zeros((nsteps, 2))
    for n in range(nsteps):
        out[n, 0] = pulse_sin2_mean(t0 + n * dt, dt, a0, omega, duration)
    return out


def pulse_sine_basis_means(nsteps: int, dt: float, n_coef: int, duration: float) -> np.ndarray:
    """(nsteps, n_coef) step means of sin((k+1) pi t / T) (library, closed form)."""
    W = np.zeros((nsteps, n_coef))
    nat.check(nat.lib().dirac_pulse_sine_basis_means(
        nsteps, dt, n_coef, duration, W.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return W


def tridiag_expm_device(alpha, beta, dt: float, lo: float, hi: float) -> np.ndarray:
    """exp(-i T dt) e_1 by the device routine (test hook)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    k = a.size
    b = np.ascontiguousarray(np.concatenate([np.asarray(beta, dtype=np.float64), [0.0]])[: max(k, 1)])
    vr, vi = np.zeros(k), np.zeros(k)
    P = ctypes.POINTER(ctypes.c_double)
    nat.check(nat.lib().dirac_debug_tridiag_expm(a.ctypes.data_as(P), b.ctypes.data_as(P), k, dt,
                                                 lo, hi, vr.ctypes.data_as(P), vi.ctypes.data_as(P)))
    return vr + 1j * vi


class BatchPropagator:
    """Many independent problems advanced together (dirac_batch_* of include/dirac.h).

    grids: list of (nx, ny, dx, dy).  All problems share mass, c, stencil
    order, boundary, precision, m_max; each has its own state, potential,
    shift and vector potential.
    """

    def __init__(self, grids, mass: float = 1.0, c: float = 137.036, order: int = 2,
                 boundary: str = "periodic", m_max: int = 20, precision: str = "fp64"):
        L = nat.lib()
        self.grids = [tuple(g) for g in grids]
        n = len(self.grids)
        nx = (ctypes.c_int * n)(*[g[0] for g in self.grids])
        ny = (ctypes.c_int * n)(*[g[1] for g in self.grids])
        dx = (ctypes.c_double * n)(*[g[2] for g in self.grids])
        dy = (ctypes.c_double * n)(*[g[3] for g in self.grids])
        b = {"periodic": nat.PERIODIC, "dirichlet": nat.DIRICHLET}[boundary]
        prec = {"fp64": nat.FP64, "mixed": nat.MIXED}[precision]
        self._b = ctypes.c_void_p()
        self._stream = _stream_ptr()
        nat.check(L.dirac_batch_create(ctypes.byref(self._b), n, nx, ny, dx, dy, mass, c, order, b,
                                       prec, m_max, self._stream))

    @property
    def n(self) -> int:
        return len(self.grids)

    def set_fields(self, problem: int, V=None, A=(0.0, 0.0), shift: float = 0.0):
        ptr = None
        if V is not None:
            torch = _torch()
            nx, ny = self.grids[problem][:2]
            if V.dtype != torch.float64 or not V.is_cuda or tuple(V.shape) != (ny, nx) \
                    or not V.is_contiguous():
                raise ValueError("V must be a contiguous CUDA float64 tensor (ny, nx)")
            ptr = ctypes.c_void_p(V.data_ptr())
        nat.check(nat.lib().dirac_batch_set_fields(self._b, problem, ptr, float(A[0]), float(A[1]),
                                                   float(shift)))

    def set_step_mode(self, mode: str = "auto"):
        """'auto', 'passes' or 'one_launch' (see dirac_batch_set_step_mode)."""
        code = {"auto": nat.STEP_AUTO, "passes": nat.STEP_PASSES, "one_launch": nat.STEP_ONE_LAUNCH}[mode]
        nat.check(nat.lib().dirac_batch_set_step_mode(self._b, code))

    def set_launch_shape(self, tile_height: int, ctas_per_sm: int = 0):
        nat.check(nat.lib().dirac_batch_set_launch_shape(self._b, tile_height, ctas_per_sm))

    def steps(self, psis, nsteps: int, dt: float, m: int, tol: float = 0.0, A=None,
              info: bool = False):
        """psis: list of CUDA complex128 tensors (ny, nx, 2); A: optional array
        (nsteps, n_problems, 2) of per-step vector potentials."""
        if len(psis) != self.n:
            raise ValueError("need one state per problem")
        for p, g in zip(psis, self.grids):
            _check_psi(p, g[1], g[0])
        ptrs = (ctypes.c_void_p * self.n)(*[p.data_ptr() for p in psis])
        a_ptr, a_arr = None, None
        if A is not None:
            a_arr = np.ascontiguousarray(A, dtype=np.float64).reshape(nsteps, self.n, 2)
            a_ptr = a_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        out = (nat.StepInfoC * self.n)() if info else None
        nat.check(nat.lib().dirac_batch_steps(self._b, ptrs, nsteps, dt, m, tol, a_ptr, out))
        return [_info(o) for o in out] if info else None

    def autotune(self, psis, dt: float, m: int, A=None, steps: int = 3) -> dict:
        """Pick the fastest launch shape (see dirac_batch_autotune); states unchanged."""
        ptrs = (ctypes.c_void_p * self.n)(*[p.data_ptr() for p in psis])
        a_ptr, a_arr = None, None
        if A is not None:
            a_arr = np.ascontiguousarray(A, dtype=np.float64).reshape(steps, self.n, 2)
            a_ptr = a_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r = nat.TuneResultC()
        nat.check(nat.lib().dirac_batch_autotune(self._b, ptrs, dt, m, a_ptr, steps, ctypes.byref(r)))
        return {"tile_height": r.tile_height, "ctas_per_sm": r.ctas_per_sm,
                "ms_per_step": r.ms_per_step, "from_cache": bool(r.from_cache),
                "candidates": r.candidates}

    def use_graphs(self, enable: bool = True):
        nat.check(nat.lib().dirac_batch_use_graphs(self._b, 1 if enable else 0))

    def sync(self):
        out = (nat.StepInfoC * self.n)()
        nat.check(nat.lib().dirac_batch_sync(self._b, out))
        return [_info(o) for o in out]

    def profile(self, enable: bool = True):
        nat.check(nat.lib().dirac_batch_profile_enable(self._b, 1 if enable else 0))

    def profile_read(self) -> dict:
        ms = (ctypes.c_double * nat.KERNEL_KINDS)()
        n = (ctypes.c_longlong * nat.KERNEL_KINDS)()
        nat.check(nat.lib().dirac_batch_profile_read(self._b, ms, n))
        return {"pass": (ms[0], n[0]), "recombine": (ms[1], n[1]), "step": (ms[2], n[2])}

    @property
    def kernel_launches(self) -> int:
        return int(nat.lib().dirac_batch_kernel_launches(self._b))

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            nat.lib().dirac_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
