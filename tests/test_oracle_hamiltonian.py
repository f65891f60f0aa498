"""Pins of the oracle's Hamiltonian (Eq. 12) against hand-derived values.

Closed forms written here from the paper's operator, not from the oracle's
code: plane-wave eigenpairs of the central stencil, individual matrix
elements, the free spectrum, and Hermiticity.
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from paper_1407_7370_gb300 import workloads as wl

C = 137.036


def plane_wave_eigpair(nx, ny, dx, dy, jx, jy, order, A, V0, mass=1.0, c=C, sign=+1):
    """psi = chi exp(i k.x) with chi the eigenvector of the 2x2 symbol; returns (psi, E)."""
    kx, ky = 2 * np.pi * jx / (nx * dx), 2 * np.pi * jy / (ny * dy)
    if order == 2:
        px, py = np.sin(kx * dx) / dx, np.sin(ky * dy) / dy
    else:
        px = (8 * np.sin(kx * dx) - np.sin(2 * kx * dx)) / (6 * dx)
        py = (8 * np.sin(ky * dy) - np.sin(2 * ky * dy)) / (6 * dy)
    # electron: p - qA = p + A
    Px, Py = px + A[0], py + A[1]
    mc2 = mass * c * c
    E = np.sqrt(mc2 ** 2 + c * c * (Px ** 2 + Py ** 2))
    # H_k = [[mc2, c(Px - iPy)], [c(Px + iPy), -mc2]] (+V0)
    if sign > 0:
        chi = np.array([E + mc2, c * (Px + 1j * Py)])
    else:
        chi = np.array([-c * (Px - 1j * Py), E + mc2])
    chi = chi / np.linalg.norm(chi)
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    X, Y = np.meshgrid(x, y, indexing="xy")
    psi = np.exp(1j * (kx * X + ky * Y))[..., None] * chi
    return psi, V0 + sign * E


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("sign", [+1, -1])
def test_plane_wave_is_eigenvector(order, sign):
    nx, ny, dx, dy = 10, 8, 0.13, 0.21
    A, V0 = (3.5, -2.25), 7.0
    for jx, jy in [(1, 0), (0, 1), (3, -2), (-4, 3), (5, 4)]:
        psi, E = plane_wave_eigpair(nx, ny, dx, dy, jx, jy, order, A, V0, sign=sign)
        op = ham.Operator(nx, ny, dx, dy, order=order, V=np.full((ny, nx), V0), A=A)
        hpsi = ham.apply(op, psi)
        assert np.max(np.abs(hpsi - E * psi)) <= 1e-10 * abs(E)


@pytest.mark.parametrize("boundary", [ham.PERIODIC, ham.DIRICHLET])
@pytest.mark.parametrize("order", [2, 4])
def test_hermitian(boundary, order):
    g = wl.Grid(9, 7, 0.1, 0.17)
    a, b = wl.random_spinor(g, 1), wl.random_spinor(g, 2)
    op = ham.Operator(9, 7, 0.1, 0.17, order=order, boundary=boundary,
                      V=wl.random_potential(g, 3), A=(1.3, -0.7))
    lhs = ham.inner(a, ham.apply(op, b))
    rhs = np.conj(ham.inner(b, ham.apply(op, a)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _element(op, row, col):
    """<row|H|col> for (j, l, component) triples."""
    e = np.zeros((op.ny, op.nx, 2), complex)
    e[col[1], col[0], col[2]] = 1.0
    return ham.apply(op, e)[row[1], row[0], row[2]]


def test_matrix_elements_order2():
    nx, ny, dx, dy, c = 7, 6, 0.1, 0.3, C
    V = np.arange(nx * ny, dtype=float).reshape(ny, nx)
    op = ham.Operator(nx, ny, dx, dy, V=V, A=(2.0, 5.0))
    j, l, U, D = 3, 2, 0, 1
    mc2 = c * c
    assert np.isclose(_element(op, (j, l, U), (j, l, U)), mc2 + V[l, j])
    assert np.isclose(_element(op, (j, l, D), (j, l, D)), -mc2 + V[l, j])
    # same-site coupling c(A_x -/+ i A_y) from c sigma.(p + A)
    assert np.isclose(_element(op, (j, l, U), (j, l, D)), c * (2.0 - 5.0j))
    assert np.isclose(_element(op, (j, l, D), (j, l, U)), c * (2.0 + 5.0j))
    # x neighbours: c sigma_x (-i D_x)
    assert np.isclose(_element(op, (j + 1, l, D), (j, l, U)), 1j * c / (2 * dx))
    assert np.isclose(_element(op, (j - 1, l, D), (j, l, U)), -1j * c / (2 * dx))
    assert np.isclose(_element(op, (j + 1, l, U), (j, l, D)), 1j * c / (2 * dx))
    # y neighbours: c sigma_y (-i D_y)
    assert np.isclose(_element(op, (j, l + 1, D), (j, l, U)), -c / (2 * dy))
    assert np.isclose(_element(op, (j, l + 1, U), (j, l, D)), c / (2 * dy))
    assert np.isclose(_element(op, (j, l - 1, U), (j, l, D)), -c / (2 * dy))
    # nothing two sites away for order 2, no same-component neighbour coupling
    assert _element(op, (j + 2, l, D), (j, l, U)) == 0
    assert _element(op, (j + 1, l, U), (j, l, U)) == 0


def test_matrix_elements_order4_and_boundaries():
    nx, ny, dx, dy, c = 8, 6, 0.1, 0.3, C
    op = ham.Operator(nx, ny, dx, dy, order=4)
    j, l = 3, 2
    assert np.isclose(_element(op, (j + 1, l, 1), (j, l, 0)), 1j * c * 8 / (12 * dx))
    assert np.isclose(_element(op, (j + 2, l, 1), (j, l, 0)), -1j * c / (12 * dx))
    assert np.isclose(_element(op, (j, l + 2, 1), (j, l, 0)), c / (12 * dy))
    # periodic wrap vs Dirichlet cut at the edge
    op2 = ham.Operator(nx, ny, dx, dy)
    assert np.isclose(_element(op2, (0, l, 1), (nx - 1, l, 0)), 1j * c / (2 * dx))
    assert np.isclose(_element(op2, (j, 0, 1), (j, ny - 1, 0)), -c / (2 * dy))
    op3 = ham.Operator(nx, ny, dx, dy, boundary=ham.DIRICHLET)
    assert _element(op3, (0, l, 1), (nx - 1, l, 0)) == 0
    assert _element(op3, (j, 0, 1), (j, ny - 1, 0)) == 0
    assert np.isclose(_element(op3, (1, l, 1), (0, l, 0)), 1j * c / (2 * dx))


@pytest.mark.parametrize("order", [2, 4])
def test_dense_spectrum_is_free_dispersion(order):
    nx, ny, dx, dy, A = 6, 4, 0.2, 0.15, (1.7, -0.4)
    op = ham.Operator(nx, ny, dx, dy, order=order, A=A)
    ev = np.linalg.eigvalsh(ham.dense(op))
    expect = []
    for jx in range(nx):
        for jy in range(ny):
            _, E = plane_wave_eigpair(nx, ny, dx, dy, jx, jy, order, A, 0.0)
            expect += [E, -E]
    assert np.allclose(np.sort(ev), np.sort(expect), rtol=0, atol=1e-9 * C * C)


# --- planted mistakes: each must be caught by the pins above --------------------

def test_pins_catch_sigma_y_sign(monkeypatch):
    monkeypatch.setattr(ham, "SIGMA_Y", -ham.SIGMA_Y)
    with pytest.raises(AssertionError):
        test_plane_wave_is_eigenvector(2, +1)


def test_pins_catch_charge_sign(monkeypatch):
    monkeypatch.setattr(ham, "CHARGE", +1.0)
    with pytest.raises(AssertionError):
        test_plane_wave_is_eigenvector(2, +1)


def test_pins_catch_axis_swap(monkeypatch):
    orig = ham.derivative
    monkeypatch.setattr(ham, "derivative", lambda f, axis, h, o, b: orig(f, 1 - axis, h, o, b))
    with pytest.raises(AssertionError):
        test_plane_wave_is_eigenvector(2, +1)


def test_pins_catch_one_sided_difference(monkeypatch):
    def forward(f, axis, h, order, boundary):
        return (ham._neighbour(f, axis, 1, boundary) - f) / h
    monkeypatch.setattr(ham, "derivative", forward)
    with pytest.raises(AssertionError):
        test_hermitian(ham.PERIODIC, 2)
