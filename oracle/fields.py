"""First-order Magnus field average over a time step (oracle; test infrastructure only).

Eq. 16 keeps the first Magnus term, exp(-i integral_t^{t+dt} H(t') dt').  H is
affine in a spatially uniform vector potential, so that integral equals
dt * H(A_mean) with A_mean the mean of A(t') over [t, t+dt].  Here the mean is
taken by Gauss-Legendre quadrature (16 nodes per smooth piece; the pulse is
split where it switches on or off), which is exact to rounding for the
smooth, slowly varying pulses used here.
"""
from __future__ import annotations

import math

import numpy as np

_NODES, _WEIGHTS = np.polynomial.legendre.leggauss(16)


def sin2_pulse(pulse, t: float) -> float:
    """A_x(t) = A0 sin^2(pi t/T) sin(omega t) on [0, T], zero outside."""
    if t < 0.0 or t > pulse.duration:
        return 0.0
    return pulse.a0 * math.sin(math.pi * t / pulse.duration) ** 2 * math.sin(pulse.omega * t)


def step_mean(pulse, t0: float, dt: float) -> float:
    """(1/dt) * integral_{t0}^{t0+dt} A_x(t) dt."""
    a, b = max(t0, 0.0), min(t0 + dt, pulse.duration)
    if b <= a:
        return 0.0
    half, mid = 0.5 * (b - a), 0.5 * (a + b)
    total = sum(w * sin2_pulse(pulse, mid + half * x) for x, w in zip(_NODES, _WEIGHTS))
    return float(total * half / dt)
