"""Closed-form propagator of the free discretised operator (oracle; test infrastructure only).

With V constant and a uniform vector potential on a periodic grid, the
discretised H of Eq. 12 is diagonal in the discrete Fourier basis.  On
exp(i k x) the central stencil -i D has the eigenvalue

    order 2: sin(k h) / h
    order 4: (8 sin(k h) - sin(2 k h)) / (6 h)

so each Fourier mode carries the 2x2 matrix

    H_k = c sigma_x (pt_x - q A_x) + c sigma_y (pt_y - q A_y) + m c^2 sigma_z + V0,

whose square (minus V0) is E_k^2 = m^2c^4 + c^2 |pt - qA|^2 times the unit
matrix -- the discrete analogue of Eq. 25.  Hence, per mode,

    exp(-i H_k dt) = exp(-i V0 dt) [cos(E_k dt) - i sin(E_k dt) / E_k (H_k - V0)].

This is the exact first-Magnus step that the Krylov step approximates, used
to pin the propagator (Sec. 6 compares to an analytic free solution likewise).
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham


def stencil_momentum(k: np.ndarray, h: float, order: int) -> np.ndarray:
    """Eigenvalue of -i D (central difference) on the plane wave exp(i k x)."""
    if order == 2:
        return np.sin(k * h) / h
    if order == 4:
        return (8.0 * np.sin(k * h) - np.sin(2.0 * k * h)) / (6.0 * h)
    raise ValueError("order must be 2 or 4")


def wavenumbers(op: ham.Operator):
    kx = 2.0 * np.pi * np.fft.fftfreq(op.nx, d=op.dx)
    ky = 2.0 * np.pi * np.fft.fftfreq(op.ny, d=op.dy)
    return np.meshgrid(kx, ky, indexing="xy")


def dispersion(op: ham.Operator) -> np.ndarray:
    """E_k >= 0 for every Fourier mode, shape (ny, nx)."""
    KX, KY = wavenumbers(op)
    px = stencil_momentum(KX, op.dx, op.order) - ham.CHARGE * op.A[0]
    py = stencil_momentum(KY, op.dy, op.order) - ham.CHARGE * op.A[1]
    mc2 = op.mass * op.c * op.c
    return np.sqrt(mc2 * mc2 + op.c * op.c * (px * px + py * py))


def step(op: ham.Operator, psi: np.ndarray, dt: float, v0: float = 0.0) -> np.ndarray:
    """exp(-i H dt) psi exactly, for V = v0 (a constant) and periodic boundaries."""
    if op.boundary != ham.PERIODIC:
        raise ValueError("closed form needs periodic boundaries")
    KX, KY = wavenumbers(op)
    px = stencil_momentum(KX, op.dx, op.order) - ham.CHARGE * op.A[0]
    py = stencil_momentum(KY, op.dy, op.order) - ham.CHARGE * op.A[1]
    mc2 = op.mass * op.c * op.c
    e = np.sqrt(mc2 * mc2 + op.c * op.c * (px * px + py * py))
    f = np.fft.fft2(psi, axes=(0, 1))
    u, d = f[..., 0], f[..., 1]
    # (H_k - V0) applied to (u, d)
    hu = mc2 * u + op.c * (px - 1j * py) * d
    hd = op.c * (px + 1j * py) * u - mc2 * d
    cs, sn = np.cos(e * dt), np.sin(e * dt) / e
    out = np.empty_like(f)
    out[..., 0] = cs * u - 1j * sn * hu
    out[..., 1] = cs * d - 1j * sn * hd
    out *= np.exp(-1j * v0 * dt)
    return np.fft.ifft2(out, axes=(0, 1))


def propagate(op: ham.Operator, psi: np.ndarray, dt: float, steps: int, pulse=None,
              t0: float = 0.0, v0: float = 0.0) -> np.ndarray:
    from . import fields
    for n in range(steps):
        if pulse is not None:
            op.A = (fields.step_mean(pulse, t0 + n * dt, dt), op.A[1])
        psi = step(op, psi, dt, v0)
    return psi
