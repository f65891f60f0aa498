"""Gradients of a final-state observable through the time-discrete propagation
(oracle; test infrastructure only).

The map differentiated is the time-discrete propagation of Sec. 4 with the
first Magnus term of Eq. 16, psi_{n+1} = exp(-i H_n dt) psi_n with
H_n = H(V, A_n) of Eq. 12 and A_n the step mean of the vector potential,
taken with the exact matrix exponential of the discretised operator (the
Krylov approximation of Eq. 17 is treated as exact; its Eq. 18 error lies far
below the tolerances of a gradient check).  Parameters: the potential energy
V at every site and the step-mean vector potential A_n = (A_x, A_y) of every
step.

Observables (real):
  "px":   <p_x> = dx dy Re <psi_N, p_x psi_N>, p_x = -i D_x with the
          Hamiltonian's own central difference
  "proj": |dx dy <phi, psi_N>|^2, the population of a fixed state phi

The gradient is defined here by forward-mode directional derivatives.  For a
parameter theta with dH_n/dtheta = E_n the step's derivative is the Frechet
derivative of the exponential, L(X, Y) = d/de exp(X + e Y) at e = 0, with
X = -i dt H_n and Y = -i dt E_n (scipy.linalg.expm_frechet):
    d psi_{n+1} = exp(X) d psi_n + L(X, Y) psi_n,
and dL = 2 Re <lambda_N, d psi_N> with lambda_N = dL/d conj(psi_N) (the
Wirtinger derivative of the real observable).  Dense matrices: tiny grids only.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from . import hamiltonian as ham


def momentum_x(op: ham.Operator, psi: np.ndarray) -> np.ndarray:
    """p_x psi = -i D_x psi (central difference of the operator's order and boundary)."""
    return -1j * ham.derivative(psi, 1, op.dx, op.order, op.boundary)


def observable(kind: str, op: ham.Operator, psi: np.ndarray, phi: np.ndarray | None = None):
    """(L, lambda_N = dL/d conj(psi)) for the observable ``kind``."""
    w = op.dx * op.dy
    if kind == "px":
        p = momentum_x(op, psi)
        return w * ham.inner(psi, p).real, w * p
    if kind == "proj":
        amp = w * ham.inner(phi, psi)
        return abs(amp) ** 2, w * amp * phi
    raise ValueError(kind)


def _op_at(op: ham.Operator, a) -> ham.Operator:
    return dataclasses.replace(op, A=(float(a[0]), float(a[1])))


def _generators(op: ham.Operator, A_steps: np.ndarray, dt: float):
    """X_n = -i dt H_n (dense) for every step."""
    return [-1j * dt * ham.dense(_op_at(op, a)) for a in np.asarray(A_steps, dtype=float)]


def forward(op: ham.Operator, psi0: np.ndarray, dt: float, A_steps) -> list:
    """[psi_0, psi_1, ..., psi_N] of the exact time-discrete map."""
    states = [np.asarray(psi0, dtype=np.complex128)]
    for X in _generators(op, A_steps, dt):
        states.append((scipy.linalg.expm(X) @ states[-1].reshape(-1)).reshape(psi0.shape))
    return states


def loss(op, psi0, dt, A_steps, kind, phi=None) -> float:
    return observable(kind, op, forward(op, psi0, dt, A_steps)[-1], phi)[0]


@dataclasses.dataclass
class Gradient:
    loss: float
    dV: np.ndarray          # dL/dV at the requested sites (flat site index order)
    dA: np.ndarray          # dL/dA_n, shape (nsteps, 2)


def _site_direction(nx: int, ny: int, site: int) -> np.ndarray:
    """dH/dV(site): the identity on both components of one site (flattened (ny, nx, 2))."""
    d = np.zeros(nx * ny * 2)
    d[2 * site] = d[2 * site + 1] = 1.0
    return np.diag(d)


def _a_direction(op: ham.Operator, comp: int) -> np.ndarray:
    """dH/dA_comp = c sigma_comp on every site (electron: p - qA = p + A)."""
    sig = ham.SIGMA_X if comp == 0 else ham.SIGMA_Y
    return -ham.CHARGE * op.c * np.kron(np.eye(op.nx * op.ny), sig)


def gradient(op: ham.Operator, psi0: np.ndarray, dt: float, A_steps, kind: str,
             phi=None, sites=None) -> Gradient:
    """dL/dV at ``sites`` (flat indices j + nx * l; all sites if None) and dL/dA_n."""
    A_steps = np.asarray(A_steps, dtype=float)
    Xs = _generators(op, A_steps, dt)
    Us = [scipy.linalg.expm(X) for X in Xs]
    states = [psi0.reshape(-1).astype(np.complex128)]
    for U in Us:
        states.append(U @ states[-1])
    L, lam = observable(kind, op, states[-1].reshape(psi0.shape), phi)
    lam = lam.reshape(-1)
    nsteps = len(Xs)

    def directional(E_of_step) -> float:
        dpsi = np.zeros_like(states[0])
        for n in range(nsteps):
            E = E_of_step(n)
            dpsi = Us[n] @ dpsi
            if E is not None:
                dpsi = dpsi + scipy.linalg.expm_frechet(Xs[n], -1j * dt * E, compute_expm=False) @ states[n]
        return 2.0 * np.vdot(lam, dpsi).real

    sites = range(op.nx * op.ny) if sites is None else sites
    dV = np.array([directional(lambda n, E=_site_direction(op.nx, op.ny, s): E) for s in sites])
    dA = np.zeros((nsteps, 2))
    for comp in (0, 1):
        E = _a_direction(op, comp)
        for m in range(nsteps):
            dA[m, comp] = directional(lambda n: E if n == m else None)
    return Gradient(L, dV, dA)


def jvp(op: ham.Operator, psi0: np.ndarray, dt: float, A_steps, kind: str, phi=None,
        dV=None, dA=None):
    """(L, directional derivative of L along (dV, dA)) in one forward-mode
    sweep: dV a field (ny, nx) added to V, dA (nsteps, 2) added to the step
    means; the step's derivative is the Frechet derivative of the exponential
    in the direction E_n = diag(dV) + dA_n . (dH/dA)."""
    A_steps = np.asarray(A_steps, dtype=float)
    Xs = _generators(op, A_steps, dt)
    n2 = 2 * op.nx * op.ny
    ev = np.zeros(n2) if dV is None else np.repeat(np.asarray(dV, dtype=float).reshape(-1), 2)
    ax, ay = _a_direction(op, 0), _a_direction(op, 1)
    psi = psi0.reshape(-1).astype(np.complex128)
    dpsi = np.zeros_like(psi)
    for n, X in enumerate(Xs):
        E = np.diag(ev).astype(np.complex128)
        if dA is not None:
            E = E + dA[n, 0] * ax + dA[n, 1] * ay
        U, F = scipy.linalg.expm_frechet(X, -1j * dt * E)
        dpsi = U @ dpsi + F @ psi
        psi = U @ psi
    L, lam = observable(kind, op, psi.reshape(psi0.shape), phi)
    return L, 2.0 * np.vdot(lam.reshape(-1), dpsi).real


def fd_gradient_V(op, psi0, dt, A_steps, kind, phi, site: int, h: float) -> float:
    """Central finite difference of L in V at one site (step h)."""
    def L_at(dv):
        V = np.zeros((op.ny, op.nx)) if op.V is None else op.V.copy()
        V.reshape(-1)[site] += dv
        return loss(dataclasses.replace(op, V=V), psi0, dt, A_steps, kind, phi)
    return (L_at(h) - L_at(-h)) / (2.0 * h)


def fd_gradient_A(op, psi0, dt, A_steps, kind, phi, step: int, comp: int, h: float) -> float:
    """Central finite difference of L in the step-mean A of one step."""
    def L_at(da):
        A = np.array(A_steps, dtype=float)
        A[step, comp] += da
        return loss(op, psi0, dt, A, kind, phi)
    return (L_at(h) - L_at(-h)) / (2.0 * h)


def sine_basis_means(nsteps: int, dt: float, n_coef: int, duration: float) -> np.ndarray:
    """W[n, k] = (1/dt) * integral over step n of sin((k+1) pi t / T): the step
    means of the pulse basis A_x(t) = sum_k a_k sin((k+1) pi t / T) (closed form)."""
    t0 = np.arange(nsteps)[:, None] * dt
    w = (np.arange(n_coef)[None, :] + 1) * np.pi / duration
    return (np.cos(w * t0) - np.cos(w * (t0 + dt))) / (w * dt)


__all__ = ["momentum_x", "observable", "forward", "loss", "gradient", "Gradient", "jvp",
           "fd_gradient_V", "fd_gradient_A", "sine_basis_means"]
