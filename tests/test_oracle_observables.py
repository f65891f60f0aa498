"""Pins of the oracle's final-state observables (``oracle/adjoint.py``:
``momentum_x`` and ``observable``) against closed forms that do not go
through finite differences of the same functions.

* <p_x> (p_x = -i D_x, Sec. 3: p = -i grad with hbar = 1).  A discrete plane
  wave psi_j = s exp(i k x_j) on a periodic grid is an eigenvector of the
  central difference: -i D_x psi = p~(k) psi with p~ = sin(k dx)/dx (order 2)
  or (8 sin(k dx) - sin(2 k dx))/(6 dx) (order 4).  Normalised so that
  dx dy sum |psi|^2 = 1, its <p_x> is exactly p~(k) and lambda = dL/d conj(psi)
  is dx dy p~(k) psi.  A superposition of plane waves of different k (which
  are orthogonal on the periodic grid) has <p_x> = sum_k w_k p~(k) with w_k
  the weights of the modes.
* |dx dy <phi, psi>|^2: with phi = psi normalised the value is 1 and lambda is
  dx dy psi; with phi orthogonal to psi both vanish; a phase on phi changes
  nothing.
A sign flip of p_x, or a dropped dx dy weight, fails these pins.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import hamiltonian as ham


def plane_wave(nx, ny, dx, dy, jx, jy, spinor):
    """Normalised discrete plane wave of mode (jx, jy): dx dy sum |psi|^2 = 1."""
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    kx = 2.0 * np.pi * jx / (nx * dx)
    ky = 2.0 * np.pi * jy / (ny * dy)
    ph = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))
    s = np.asarray(spinor, dtype=np.complex128)
    psi = ph[..., None] * s[None, None, :]
    psi /= np.sqrt(dx * dy * np.sum(np.abs(psi) ** 2))
    return psi, kx


def p_tilde(k, h, order):
    if order == 2:
        return np.sin(k * h) / h
    return (8.0 * np.sin(k * h) - np.sin(2.0 * k * h)) / (6.0 * h)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("jx", [1, 3, -2, 7])
def test_px_of_a_plane_wave_is_the_stencil_momentum(order, jx):
    nx, ny, dx, dy = 16, 12, 0.3, 0.25
    psi, kx = plane_wave(nx, ny, dx, dy, jx, 2, (0.6 - 0.2j, 0.3 + 0.7j))
    op = ham.Operator(nx, ny, dx, dy, order=order)
    L, lam = adj.observable("px", op, psi)
    want = p_tilde(kx, dx, order)
    assert abs(L - want) <= 1e-12 * max(1.0, abs(want)), (L, want)
    np.testing.assert_allclose(lam, dx * dy * want * psi, rtol=0, atol=1e-12 * np.abs(psi).max())


def test_px_of_a_superposition_weights_the_modes():
    nx, ny, dx, dy = 20, 10, 0.2, 0.2
    a, kxa = plane_wave(nx, ny, dx, dy, 2, 0, (1.0, 0.0))
    b, kxb = plane_wave(nx, ny, dx, dy, -5, 1, (0.0, 1.0j))
    c, kxc = plane_wave(nx, ny, dx, dy, 4, 3, (0.5, -0.5))
    w = np.array([0.5, 0.3, 0.2])
    psi = np.sqrt(w[0]) * a + np.sqrt(w[1]) * b + np.sqrt(w[2]) * c   # dx dy sum |psi|^2 = 1
    op = ham.Operator(nx, ny, dx, dy)
    L, _ = adj.observable("px", op, psi)
    want = float(np.dot(w, [p_tilde(k, dx, 2) for k in (kxa, kxb, kxc)]))
    assert abs(L - want) <= 1e-12 * abs(want) + 1e-13, (L, want)


def test_px_is_real_for_any_state():
    """p_x is Hermitian on the periodic grid: <psi, p_x psi> has no imaginary part."""
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((9, 11, 2)) + 1j * rng.standard_normal((9, 11, 2))
    op = ham.Operator(11, 9, 0.1, 0.1, order=4)
    val = ham.inner(psi, adj.momentum_x(op, psi))
    assert abs(val.imag) <= 1e-12 * abs(val), val


def test_proj_of_the_state_itself_is_one():
    nx, ny, dx, dy = 12, 10, 0.15, 0.2
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((ny, nx, 2)) + 1j * rng.standard_normal((ny, nx, 2))
    psi /= np.sqrt(dx * dy * np.sum(np.abs(psi) ** 2))
    op = ham.Operator(nx, ny, dx, dy)
    L, lam = adj.observable("proj", op, psi, phi=psi)
    assert abs(L - 1.0) <= 1e-13
    np.testing.assert_allclose(lam, dx * dy * psi, rtol=0, atol=1e-14 * np.abs(psi).max())
    # a phase on phi changes neither the population nor lambda's modulus
    L2, lam2 = adj.observable("proj", op, psi, phi=np.exp(0.7j) * psi)
    assert abs(L2 - 1.0) <= 1e-13
    np.testing.assert_allclose(np.abs(lam2), dx * dy * np.abs(psi), rtol=1e-12)


def test_proj_of_an_orthogonal_state_vanishes():
    nx, ny, dx, dy = 14, 8, 0.2, 0.2
    a, _ = plane_wave(nx, ny, dx, dy, 1, 0, (1.0, 0.5))
    b, _ = plane_wave(nx, ny, dx, dy, 3, 1, (0.2, 1.0))
    op = ham.Operator(nx, ny, dx, dy)
    L, lam = adj.observable("proj", op, a, phi=b)
    assert abs(L) <= 1e-26
    assert np.abs(lam).max() <= 1e-13
    # half and half: population 1/2
    L, _ = adj.observable("proj", op, (a + b) / np.sqrt(2.0), phi=a)
    assert abs(L - 0.5) <= 1e-13


def test_planted_sign_flip_of_px_fails_the_plane_wave_pin(monkeypatch):
    nx, ny, dx, dy = 16, 12, 0.3, 0.25
    psi, kx = plane_wave(nx, ny, dx, dy, 3, 1, (1.0, 0.2j))
    op = ham.Operator(nx, ny, dx, dy)
    want = p_tilde(kx, dx, 2)
    flipped = lambda o, f: 1j * ham.derivative(f, 1, o.dx, o.order, o.boundary)  # noqa: E731
    monkeypatch.setattr(adj, "momentum_x", flipped)
    L, _ = adj.observable("px", op, psi)
    assert abs(L - want) > 0.5 * abs(want)


def test_planted_missing_weight_fails_the_projection_pin(monkeypatch):
    nx, ny, dx, dy = 12, 10, 0.15, 0.2
    psi, _ = plane_wave(nx, ny, dx, dy, 2, 2, (1.0, 1.0))
    op = ham.Operator(nx, ny, dx, dy)
    real = adj.observable

    def unweighted(kind, o, p, phi=None):
        if kind == "proj":
            amp = ham.inner(phi, p)
            return abs(amp) ** 2, amp * phi
        return real(kind, o, p, phi)

    monkeypatch.setattr(adj, "observable", unweighted)
    L, _ = adj.observable("proj", op, psi, phi=psi)
    assert abs(L - 1.0) > 0.5
