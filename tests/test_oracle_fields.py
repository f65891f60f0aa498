"""Pin of the oracle's Magnus-1 field mean against the closed-form integral."""
import math

import pytest

from oracle import fields
from paper_1407_7370_gb300 import workloads as wl


def closed_form_mean(p, t0, dt):
    """sin^2(pi t/T) sin(w t) = sin(wt)/2 - sin((w+W)t)/4 - sin((w-W)t)/4, W = 2 pi/T."""
    a, b = max(t0, 0.0), min(t0 + dt, p.duration)
    if b <= a:
        return 0.0
    W = 2 * math.pi / p.duration

    def integ(nu):  # (cos(nu a) - cos(nu b)) / nu without cancellation
        return 2.0 * math.sin(0.5 * nu * (a + b)) * math.sin(0.5 * nu * (b - a)) / nu
    return p.a0 * (0.5 * integ(p.omega) - 0.25 * integ(p.omega + W) - 0.25 * integ(p.omega - W)) / dt


@pytest.mark.parametrize("t0", [-1e-4, 0.0, 0.1234, 0.5, 0.9999, 1.0, 2.0])
def test_step_mean_matches_closed_form(t0):
    p = wl.SinSquaredPulse(50.0, 0.05, 1.0)
    dt = 2e-4
    ref = closed_form_mean(p, t0, dt)
    assert abs(fields.step_mean(p, t0, dt) - ref) <= 1e-13 * p.a0


def test_long_step_mean():
    p = wl.SinSquaredPulse(50.0, 3.0, 1.0)
    assert abs(fields.step_mean(p, 0.2, 0.05) - closed_form_mean(p, 0.2, 0.05)) <= 1e-11
