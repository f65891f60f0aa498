"""Discretised 2D Dirac Hamiltonian (oracle; test infrastructure only).

Sec. 3, Eq. 12 in two dimensions with two-component spinors:

    H = c * sum_i alpha_i (p_i - q A_i) + beta m c^2 + q phi,
    alpha_1 = sigma_x, alpha_2 = sigma_y, beta = sigma_z   (Sec. 3),

with p_i = -i d/dx_i (hbar = 1), electron charge q = -1 and V = q phi the
potential energy.  The vector potential is uniform in space (one value per
time step, the dipole approximation).  Derivatives are finite differences on
a uniform grid (Sec. 7); they are read as *central* first-derivative stencils
so that -i d/dx stays Hermitian, which Sec. 8 requires of the discretisation:

    order 2: (f[j+1] - f[j-1]) / (2h)
    order 4: (-f[j+2] + 8 f[j+1] - 8 f[j-1] + f[j-2]) / (12h)

Boundaries are periodic, or Dirichlet (the field is zero outside the grid).
Spinor fields are complex128 arrays of shape (ny, nx, 2): axis 0 is y, axis 1
is x, axis 2 the (upper, lower) component.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SIGMA_X = np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)
SIGMA_Y = np.array([[0.0, -1.0j], [1.0j, 0.0]], dtype=np.complex128)
SIGMA_Z = np.array([[1.0, 0.0], [0.0, -1.0]], dtype=np.complex128)
CHARGE = -1.0  # the electron

PERIODIC = 0
DIRICHLET = 1


@dataclasses.dataclass
class Operator:
    """Everything that defines H for one time step."""

    nx: int
    ny: int
    dx: float
    dy: float
    mass: float = 1.0
    c: float = 137.036
    order: int = 2
    boundary: int = PERIODIC
    V: np.ndarray | None = None   # potential energy q*phi, (ny, nx), or None for 0
    A: tuple = (0.0, 0.0)         # uniform vector potential (A_x, A_y)
    shift: float = 0.0            # constant energy subtracted: H - shift


def _neighbour(f: np.ndarray, axis: int, offset: int, boundary: int) -> np.ndarray:
    """g[..., j, ...] = f[..., j + offset, ...] with the chosen boundary."""
    g = np.roll(f, -offset, axis=axis)
    if boundary == DIRICHLET:
        n = f.shape[axis]
        idx = [slice(None)] * f.ndim
        if offset > 0:
            idx[axis] = slice(n - offset, n)
        else:
            idx[axis] = slice(0, -offset)
        g[tuple(idx)] = 0.0
    return g


def derivative(f: np.ndarray, axis: int, h: float, order: int, boundary: int) -> np.ndarray:
    """Central finite-difference first derivative along ``axis``."""
    nb = lambda k: _neighbour(f, axis, k, boundary)  # noqa: E731
    if order == 2:
        return (nb(1) - nb(-1)) / (2.0 * h)
    if order == 4:
        return (-nb(2) + 8.0 * nb(1) - 8.0 * nb(-1) + nb(-2)) / (12.0 * h)
    raise ValueError("order must be 2 or 4")


def pauli(sigma: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 2x2 matrix to the spinor at every site."""
    return np.einsum("ab,...b->...a", sigma, psi)


def apply(op: Operator, psi: np.ndarray) -> np.ndarray:
    """(H - shift) psi, Eq. 12."""
    mc2 = op.mass * op.c * op.c
    # kinetic momenta (p_i - q A_i) psi, p_i = -i d/dx_i
    pi_x = -1j * derivative(psi, 1, op.dx, op.order, op.boundary) - CHARGE * op.A[0] * psi
    pi_y = -1j * derivative(psi, 0, op.dy, op.order, op.boundary) - CHARGE * op.A[1] * psi
    out = op.c * (pauli(SIGMA_X, pi_x) + pauli(SIGMA_Y, pi_y)) + mc2 * pauli(SIGMA_Z, psi)
    if op.V is not None:
        out = out + op.V[..., None] * psi
    if op.shift != 0.0:
        out = out - op.shift * psi
    return out


def dense(op: Operator) -> np.ndarray:
    """The full matrix of (H - shift) on the flattened (ny, nx, 2) index; tiny grids only."""
    n = op.nx * op.ny * 2
    cols = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[:] = 0.0
        e[k] = 1.0
        cols[:, k] = apply(op, e.reshape(op.ny, op.nx, 2)).reshape(n)
    return cols


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum over sites and components of conj(a) b (no grid weight)."""
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def norm(a: np.ndarray) -> float:
    return float(np.sqrt(np.vdot(a.reshape(-1), a.reshape(-1)).real))
