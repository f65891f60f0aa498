"""Pins of the oracle's gradients (forward-mode Frechet derivatives of the exact
time-discrete map) against what does not share their route:

* central finite differences of the forward map itself;
* invariances: a uniform change of V only multiplies psi_N by a phase, so its
  total derivative vanishes for both observables; without a potential and
  with periodic boundaries p_x commutes with every H_n, so <p_x> does not
  depend on the vector potential;
* the closed-form step means of the sine basis of the pulse.
A planted sign error in the Frechet direction fails the finite-difference pin.
"""
import dataclasses

import numpy as np
import pytest
import scipy.linalg

from oracle import adjoint as adj
from oracle import hamiltonian as ham
from paper_1407_7370_gb300 import workloads as wl

C = 137.036


def small_case(nx=6, ny=5, dx=0.4, z=2.0, seed=3):
    g = wl.Grid(nx, ny, dx, dx)
    V = wl.soft_core(g, z) + 0.3 * wl.random_potential(g, seed, scale=1.0)
    op = ham.Operator(nx, ny, dx, dx, V=V, shift=C * C)
    psi0 = wl.positive_energy_packet(g, p0=(2.0, 1.0), sigma_x=0.8)
    phi = wl.normalise(wl.random_spinor(g, seed + 1), g)
    A = np.array([[0.5, -0.2], [1.0, 0.3], [-0.7, 0.1], [0.2, 0.4]])
    return op, psi0, phi, A


@pytest.mark.parametrize("kind", ["px", "proj"])
def test_gradient_matches_central_differences(kind):
    op, psi0, phi, A = small_case()
    dt = 2e-4
    sites = [0, 7, 13, 29]
    g = adj.gradient(op, psi0, dt, A, kind, phi, sites=sites)
    for s, d in zip(sites, g.dV):
        fd = adj.fd_gradient_V(op, psi0, dt, A, kind, phi, s, 1e-4)
        assert abs(d - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(g.loss)), (s, d, fd)
    for n in range(A.shape[0]):
        for comp in (0, 1):
            fd = adj.fd_gradient_A(op, psi0, dt, A, kind, phi, n, comp, 1e-4)
            assert abs(g.dA[n, comp] - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(g.loss)), (n, comp)


@pytest.mark.parametrize("kind", ["px", "proj"])
def test_directional_derivative_matches_central_differences(kind):
    """One forward-mode sweep along a random (dV, dA) against the central
    difference of the forward map along the same direction."""
    op, psi0, phi, A = small_case()
    dt = 2e-4
    rng = np.random.default_rng(11)
    dV = rng.standard_normal((op.ny, op.nx))
    dA = rng.standard_normal(A.shape)
    L, d = adj.jvp(op, psi0, dt, A, kind, phi, dV=dV, dA=dA)
    h = 1e-4

    def L_at(e):
        o = dataclasses.replace(op, V=op.V + e * dV)
        return adj.loss(o, psi0, dt, A + e * dA, kind, phi)
    fd = (L_at(h) - L_at(-h)) / (2 * h)
    assert abs(L - adj.loss(op, psi0, dt, A, kind, phi)) <= 1e-13 * abs(L)
    assert abs(d - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(L)), (d, fd)


@pytest.mark.parametrize("kind", ["px", "proj"])
def test_uniform_potential_changes_only_the_phase(kind):
    op, psi0, phi, A = small_case()
    g = adj.gradient(op, psi0, 2e-4, A, kind, phi)
    assert abs(g.dV.sum()) <= 1e-9 * np.sum(np.abs(g.dV))
    assert np.sum(np.abs(g.dV)) > 0


def test_free_momentum_does_not_depend_on_the_vector_potential():
    g = wl.Grid(6, 6, 0.4, 0.4)
    op = ham.Operator(6, 6, 0.4, 0.4, shift=C * C)
    psi0 = wl.positive_energy_packet(g, p0=(2.0, 0.0), sigma_x=0.8) + 0.05 * wl.random_spinor(g, 2)
    A = np.array([[3.0, 0.0], [-1.0, 2.0], [0.5, 0.5]])
    grad = adj.gradient(op, psi0, 2e-4, A, "px", sites=[0, 5])
    assert np.max(np.abs(grad.dA)) <= 1e-9 * abs(grad.loss)


def test_sine_basis_means_closed_form():
    dt, T = 0.01, 0.37
    W = adj.sine_basis_means(5, dt, 3, T)
    nodes, weights = np.polynomial.legendre.leggauss(20)
    for n in range(5):
        for k in range(3):
            t = n * dt + 0.5 * dt * (nodes + 1)
            mean = 0.5 * np.sum(weights * np.sin((k + 1) * np.pi * t / T))
            assert abs(W[n, k] - mean) <= 1e-14


def test_pins_catch_a_sign_error_in_the_frechet_direction(monkeypatch):
    real = scipy.linalg.expm_frechet

    def flipped(X, E, **kw):
        return real(X, -E, **kw)
    monkeypatch.setattr(adj.scipy.linalg, "expm_frechet", flipped)
    with pytest.raises(AssertionError):
        test_gradient_matches_central_differences("proj")
