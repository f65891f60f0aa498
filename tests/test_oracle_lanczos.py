"""Pins of the oracle's Lanczos recurrence, Krylov step and eigen mode.

Against library routines (scipy expm / eigh), the closed-form free
propagator, the Lanczos relation (Eq. 5), the invariants of the Krylov step
(norm and energy), and breakdown on an exact eigenvector.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import hamiltonian as ham
from oracle import lanczos as lz
from oracle import free
from paper_1407_7370_gb300 import workloads as wl

C = 137.036


def random_hermitian(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (a + a.conj().T) / 2


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_tridiag_expm_matches_scipy_expm(k):
    rng = np.random.default_rng(k)
    alpha, beta = 3 * rng.standard_normal(k), np.abs(rng.standard_normal(k))
    T = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    ref = scipy.linalg.expm(-1j * T)[:, 0]
    assert np.allclose(lz.tridiag_expm_e1(alpha, beta), ref, atol=1e-13)


def test_lanczos_relation_and_orthogonality():
    n, k = 60, 12
    A = random_hermitian(n, 5)
    b = np.random.default_rng(6).standard_normal(n) + 0j
    res = lz.lanczos(lambda v: A @ v, b, k)
    Q = np.stack(res.q, axis=1)
    T = np.diag(res.alpha) + np.diag(res.beta[:-1], 1) + np.diag(res.beta[:-1], -1)
    R = A @ Q - Q @ T   # Eq. 5: only the last column, of norm beta_k, survives
    scale = np.linalg.norm(A, 2)
    assert np.linalg.norm(R[:, :-1]) <= 1e-12 * scale
    assert abs(np.linalg.norm(R[:, -1]) - res.beta[-1]) <= 1e-12 * scale
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) <= 1e-12
    assert np.allclose(Q[:, 0], b / np.linalg.norm(b))


def test_full_krylov_reproduces_spectrum():
    n = 10
    A = random_hermitian(n, 7)
    b = np.random.default_rng(8).standard_normal(n) + 1j
    res = lz.lanczos(lambda v: A @ v, b, n)
    T = np.diag(res.alpha) + np.diag(res.beta[:-1], 1) + np.diag(res.beta[:-1], -1)
    assert np.allclose(np.linalg.eigvalsh(T), np.linalg.eigvalsh(A), atol=1e-10)
    assert res.beta[-1] <= 1e-9


def _tiny_op(order=2, boundary=ham.PERIODIC, with_v=True):
    g = wl.Grid(6, 5, 0.1, 0.12)
    V = wl.random_potential(g, 11, scale=30.0) if with_v else None
    return g, ham.Operator(6, 5, 0.1, 0.12, order=order, boundary=boundary, V=V, A=(4.0, -2.0))


@pytest.mark.parametrize("order,boundary", [(2, ham.PERIODIC), (4, ham.PERIODIC), (2, ham.DIRICHLET)])
def test_step_matches_dense_expm(order, boundary):
    g, op = _tiny_op(order, boundary)
    psi = wl.random_spinor(g, 12)
    dt = 1e-4
    ref = (scipy.linalg.expm(-1j * dt * ham.dense(op)) @ psi.reshape(-1)).reshape(psi.shape)
    out, info = lz.krylov_step(op, psi, dt, m=30)
    assert lz.rel_l2(out, ref) <= 1e-12
    out8, info8 = lz.krylov_step(op, psi, dt, m=8)
    err8 = ham.norm(out8 - ref)
    # Eq. 18 is an estimate, loose in the paper's experience: same order or above
    assert err8 > 1e-14 and info8.err_est >= 0.1 * err8 and info8.err_est <= 1e3 * err8


@pytest.mark.parametrize("shift", [0.0, 137.036 ** 2])
def test_backward_step_matches_dense_expm(shift):
    """dt < 0 (the adjoint's backward propagation): exp(+i H |dt|) psi."""
    g, op = _tiny_op(4, ham.DIRICHLET)
    op.shift = shift
    psi = wl.random_spinor(g, 14)
    dt = -1e-4
    h = ham.dense(op) + shift * np.eye(2 * g.nx * g.ny)     # H itself: the shift only changes a phase
    ref = (scipy.linalg.expm(-1j * dt * h) @ psi.reshape(-1)).reshape(psi.shape)
    out, info = lz.krylov_step(op, psi, dt, m=30)
    assert lz.rel_l2(out, ref) <= 1e-12


def test_step_with_shift_equals_unshifted():
    g, op = _tiny_op()
    psi = wl.random_spinor(g, 13)
    a, _ = lz.krylov_step(op, psi, 1e-4, m=12)
    op.shift = C * C
    b, _ = lz.krylov_step(op, psi, 1e-4, m=12)
    assert lz.rel_l2(b, a) <= 1e-12


def test_breakdown_on_eigenvector_gives_exact_phase():
    from tests.test_oracle_hamiltonian import plane_wave_eigpair
    nx, ny, dx, dy = 8, 8, 0.1, 0.1
    psi, E = plane_wave_eigpair(nx, ny, dx, dy, 2, 1, 2, (3.0, 0.0), 0.0)
    op = ham.Operator(nx, ny, dx, dy, A=(3.0, 0.0))
    out, info = lz.krylov_step(op, psi, 1e-4, m=10)
    assert info.k_used == 1 and info.breakdown
    assert np.max(np.abs(out - np.exp(-1j * E * 1e-4) * psi)) <= 1e-13


def test_norm_and_energy_conserved_static_fields():
    g = wl.Grid(32, 32, 0.1, 0.1)
    psi = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    V = wl.smoothed_coulomb(g, 2.0, 0.5)
    op = ham.Operator(32, 32, 0.1, 0.1, V=V, A=(5.0, 0.0))
    n0, e0 = ham.norm(psi), lz.energy(op, psi)
    out, infos = lz.propagate(op, psi, 1e-4, m=10, steps=10)
    assert abs(ham.norm(out) - n0) <= 1e-13 * n0
    assert abs(lz.energy(op, out) - e0) <= 1e-12 * abs(e0)
    assert abs(infos[0].energy - e0) <= 1e-12 * abs(e0)


@pytest.mark.parametrize("order", [2, 4])
def test_packet_matches_closed_form_free_propagation(order):
    g = wl.Grid(64, 64, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    op = ham.Operator(64, 64, 0.1, 0.1, order=order, A=(20.0, 0.0))
    out, infos = lz.propagate(op, psi0.copy(), 1e-4, m=10, steps=10)
    ref = free.propagate(ham.Operator(64, 64, 0.1, 0.1, order=order, A=(20.0, 0.0)),
                         psi0.copy(), 1e-4, 10)
    err = ham.norm(out - ref)
    cumulative = sum(i.err_est for i in infos)          # Sec. 6 cumulative bound
    assert err <= max(cumulative, 1e-13 * ham.norm(ref)) + 1e-12 * ham.norm(ref)
    assert err <= 1e-11 * ham.norm(ref)


def test_tolerance_stops_early():
    g = wl.Grid(32, 32, 0.1, 0.1)
    psi = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    op = ham.Operator(32, 32, 0.1, 0.1)
    full, _ = lz.krylov_step(op, psi, 1e-4, m=20)
    out, info = lz.krylov_step(op, psi, 1e-4, m=20, tol=1e-9)
    assert 1 < info.k_used < 20 and not info.breakdown
    assert ham.norm(out - full) <= 10 * 1e-9 * ham.norm(psi)


def test_free_step_matches_dense_expm():
    for order in (2, 4):
        op = ham.Operator(6, 4, 0.2, 0.15, order=order, A=(1.7, -0.4))
        psi = wl.random_spinor(wl.Grid(6, 4, 0.2, 0.15), 21)
        ref = (scipy.linalg.expm(-1j * 3e-4 * (ham.dense(op) + 2.5 * np.eye(48)))
               @ psi.reshape(-1)).reshape(psi.shape)
        assert np.allclose(free.step(op, psi, 3e-4, v0=2.5), ref, atol=1e-12)


def test_eigs_free_spectrum_closed_form():
    op = ham.Operator(8, 8, 0.3, 0.3, A=(0.0, 0.0))
    E = np.unique(np.round(free.dispersion(op), 9))
    start = wl.random_spinor(wl.Grid(8, 8, 0.3, 0.3), 31)
    res = lz.lanczos_eigs(op, start, n_want=3, max_iter=128, tol=1e-10,
                          window=(0.0, 2 * C * C))
    assert res.values.size >= 3
    for v in res.values:
        assert np.min(np.abs(E - v)) <= 1e-6 * v


def test_eigs_matches_dense_eigh_soft_core():
    g = wl.Grid(12, 12, 0.3, 0.3)
    op = ham.Operator(12, 12, 0.3, 0.3, V=wl.soft_core(g, 2.0), shift=C * C)
    ev = np.linalg.eigvalsh(ham.dense(op))
    start = wl.positive_energy_packet(g, p0=(0.0, 0.0)) + 1e-3 * wl.random_spinor(g, 4)
    res = lz.lanczos_eigs(op, start, n_want=4, max_iter=288, tol=1e-9, window=(-C * C, 0.0))
    assert res.values.size >= 4
    for v, bnd in zip(res.values, res.bounds):
        assert np.min(np.abs(ev - v)) <= max(bnd, 1e-9)


def test_pins_catch_dropped_three_term(monkeypatch):
    """A Lanczos that forgets the -beta q_{i-1} term must fail the relation pin."""
    def broken(apply_a, b, k, stop=None):
        q = [b / ham.norm(b)]
        alpha, beta = [], []
        z = apply_a(q[0])
        for i in range(k):
            a = ham.inner(q[i], z).real
            z = z - a * q[i]
            bt = ham.norm(z)
            alpha.append(a); beta.append(bt)
            if i + 1 == k:
                break
            q.append(z / bt)
            z = apply_a(q[i + 1])
        return lz.LanczosResult(q, np.array(alpha), np.array(beta), False)
    monkeypatch.setattr(lz, "lanczos", broken)
    with pytest.raises(AssertionError):
        test_lanczos_relation_and_orthogonality()
