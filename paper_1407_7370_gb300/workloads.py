"""Seeded synthetic inputs for the Dirac Lanczos propagator.

This module only *generates inputs*: grids, initial wave packets, potentials,
pulse parameters and random test vectors.  It holds none of the propagator's
arithmetic (no finite-difference operator, no Lanczos recurrence, no matrix
exponential, no field quadrature), so that the CUDA path and the CPU oracle can
both consume the same inputs without sharing any of the method.

Workloads follow the paper's set-ups:

* Sec. 7 (Fig. 7): a free 2D packet built as a Gaussian superposition of
  positive-energy free-particle states with a mean momentum and a momentum
  width.  The positive-energy spinors are the *continuum* free-particle states
  of the Dirac equation (Sec. 3 with Eq. 25's dispersion), not eigenvectors of
  the discretised operator, so nothing here depends on the stencil.
* Sec. 5.1 (Eq. 19): the soft-core potential, and the smoothed Coulomb
  potential -Z/sqrt(r^2+a^2) used for the eigenvalue workloads.
* A linearly polarised pulse A_x(t) = A0 sin^2(pi t/T) sin(omega t) on [0, T].

Atomic units throughout (hbar = m_e = e = 1, c = 137.036).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 137.036
MASS = 1.0


@dataclasses.dataclass(frozen=True)
class Grid:
    """Uniform nx-by-ny grid; site (j, l) sits at x=(j-nx/2)dx, y=(l-ny/2)dy.

    Arrays over the grid are indexed [l, j] (y slowest, x fastest); a spinor
    field is complex128 of shape (ny, nx, 2) holding (upper, lower) components
    per site.
    """

    nx: int
    ny: int
    dx: float
    dy: float

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny

    def coords(self):
        x = (np.arange(self.nx) - self.nx // 2) * self.dx
        y = (np.arange(self.ny) - self.ny // 2) * self.dy
        return np.meshgrid(x, y, indexing="xy")  # each (ny, nx)


@dataclasses.dataclass(frozen=True)
class SinSquaredPulse:
    """A_x(t) = A0 sin^2(pi t / T) sin(omega t) for 0 <= t <= T, zero outside."""

    a0: float
    omega: float
    duration: float


def positive_energy_packet(grid: Grid, p0=(10.0, 0.0), sigma_x: float = 1.0,
                           mass: float = MASS, c: float = C_LIGHT) -> np.ndarray:
    """Gaussian superposition of positive-energy free-particle states.

    Momentum amplitude exp(-|p-p0|^2 sigma_x^2) (position-space width sigma_x,
    momentum width 1/(2 sigma_x)) times the continuum positive-energy spinor
    (E+mc^2, c(px+i py)) / sqrt(2E(E+mc^2)), E = sqrt(m^2c^4 + c^2 p^2)
    (Eq. 25).  The packet is centred on x=y=0 of the grid and normalised to
    sum |psi|^2 dx dy = 1.  Returns complex128 (ny, nx, 2).
    """
    kx = 2.0 * np.pi * np.fft.fftfreq(grid.nx, d=grid.dx)
    ky = 2.0 * np.pi * np.fft.fftfreq(grid.ny, d=grid.dy)
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    mc2 = mass * c * c
    energy = np.sqrt(mc2 * mc2 + (c * c) * (KX * KX + KY * KY))
    amp = np.exp(-((KX - p0[0]) ** 2 + (KY - p0[1]) ** 2) * sigma_x ** 2)
    norm = 1.0 / np.sqrt(2.0 * energy * (energy + mc2))
    spec = np.empty((grid.ny, grid.nx, 2), dtype=np.complex128)
    # the grid's x=0 is at index nx//2: shift the plane waves accordingly
    shift = np.exp(1j * (KX * (grid.nx // 2) * grid.dx + KY * (grid.ny // 2) * grid.dy))
    spec[..., 0] = amp * (energy + mc2) * norm * shift
    spec[..., 1] = amp * c * (KX + 1j * KY) * norm * shift
    psi = np.fft.ifft2(spec, axes=(0, 1))
    return normalise(psi, grid)


def normalise(psi: np.ndarray, grid: Grid) -> np.ndarray:
    """Scale psi so that sum |psi|^2 dx dy = 1."""
    n2 = float(np.sum(np.abs(psi) ** 2)) * grid.dx * grid.dy
    return psi / math.sqrt(n2)


def smoothed_coulomb(grid: Grid, z: float, a: float) -> np.ndarray:
    """Potential energy V = -Z / sqrt(r^2 + a^2) of an electron (float64, (ny, nx))."""
    x, y = grid.coords()
    return -z / np.sqrt(x * x + y * y + a * a)


def soft_core(grid: Grid, z: float) -> np.ndarray:
    """Eq. 19: V = -(3/2) Z / sqrt(r^2 + 3/Z^2) (float64, (ny, nx))."""
    x, y = grid.coords()
    return -1.5 * z / np.sqrt(x * x + y * y + 3.0 / (z * z))


def random_spinor(grid: Grid, seed: int) -> np.ndarray:
    """Seeded complex normal spinor field (ny, nx, 2)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((grid.ny, grid.nx, 2))
            + 1j * rng.standard_normal((grid.ny, grid.nx, 2)))


def random_potential(grid: Grid, seed: int, scale: float = 50.0) -> np.ndarray:
    """Seeded smooth-ish random potential energy (float64, (ny, nx))."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((grid.ny, grid.nx))


# ----------------------------------------------------------------------------
# The propagation workloads (sizes, physics parameters).  The oracle-sized case
# and the bandwidth-sized laser case; both use the packet above.
# ----------------------------------------------------------------------------

FREE_PACKET_64 = dict(
    name="free packet 64x64, dx=0.1, m=10, dt=1e-4, 100 steps",
    grid=Grid(64, 64, 0.1, 0.1), p0=(10.0, 0.0), sigma_x=1.0, m=10, dt=1e-4,
    steps=100, pulse=None, order=2)

LASER_PACKET_1024 = dict(
    name="laser packet 1024x1024, dx=0.05, m=20, dt=2e-4, 5000 steps",
    grid=Grid(1024, 1024, 0.05, 0.05), p0=(10.0, 0.0), sigma_x=1.0, m=20,
    dt=2e-4, steps=5000, pulse=SinSquaredPulse(50.0, 0.05, 1.0), order=2)


def batch_packets(n: int = 256, seed: int = 0, sides=(128, 256, 384, 512), dx: float = 0.05):
    """The batched workload: n packets on square grids drawn uniformly from
    `sides`, mean momenta p0 = (U[0, 50], 0) au and laser amplitudes
    A0 = U[0, 100] au (each packet in A0 sin^2(pi t) sin(0.05 t)), seeded.
    Returns (grids, p0s, a0s)."""
    rng = np.random.default_rng(seed)
    s = rng.choice(np.asarray(sides), size=n)
    p0s = rng.uniform(0.0, 50.0, size=n)
    a0s = rng.uniform(0.0, 100.0, size=n)
    grids = [Grid(int(k), int(k), dx, dx) for k in s]
    return grids, p0s, a0s


BATCH_256 = dict(
    name="256 packets on 128^2..512^2 grids, dx=0.05, m=16, dt=2e-4, 2000 steps",
    n=256, m=16, dt=2e-4, steps=2000, pulse=SinSquaredPulse(1.0, 0.05, 1.0))
