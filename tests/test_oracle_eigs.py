"""Pins of the oracle's eigenvalue mode beyond the dense-spectrum checks.

* shift-folded mode against dense eigh (the eigenvalues nearest the fold);
* Ritz vectors: the residual identity ||A a_i - theta_i a_i|| = |beta_k t_i^k|
  that accompanies the Eq. 9 bound (Sec. 2), and Eq. 8 against dense
  eigenvectors;
* breakdown on a start vector inside a 3-dimensional invariant subspace:
  three iterations, the exact closed-form energies (free dispersion, Eq. 25
  on the lattice);
* loss of orthogonality: ghost copies without reorthogonalisation, none with
  it (every converged value pairs with its own dense eigenvalue).
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import lanczos as lz
from paper_1407_7370_gb300 import workloads as wl
from test_oracle_hamiltonian import plane_wave_eigpair

C = 137.036


def soft_core_op(n=12, dx=0.3, z=2.0):
    g = wl.Grid(n, n, dx, dx)
    return g, ham.Operator(n, n, dx, dx, V=wl.soft_core(g, z), shift=C * C)


def test_folded_mode_matches_dense_eigh():
    g, op = soft_core_op(10, 0.3, 3.0)
    ev = np.linalg.eigvalsh(ham.dense(op))
    sigma = -2.0                                  # inside the gap, near the bound states
    start = wl.random_spinor(g, 5)
    res = lz.lanczos_eigs(op, start, n_want=3, max_iter=200, tol=1e-9, window=None,
                          fold=sigma)
    want = np.sort(ev[np.argsort(np.abs(ev - sigma))[:3]])
    assert res.values.size == 3
    assert np.all(np.diff(res.values) >= 0)
    # folding squares the operator: T's eigenvalues carry a rounding error of
    # about u ||A||, u ||A|| / (2 sqrt(theta)) in lambda, beside the Eq. 9 bound
    norm_a = np.max((ev - sigma) ** 2)
    for v, bnd, w in zip(res.values, res.bounds, want):
        assert abs(v - w) <= bnd + 2.2e-16 * norm_a / abs(w - sigma)
        assert abs(v - w) <= 1e-6


def test_folded_sign_comes_from_the_rayleigh_quotient():
    """With the fold between two bound states, one on each side, only the
    Rayleigh-quotient sign puts each on its side (not midway: there the two
    folded eigenvalues coincide and no Ritz vector separates them)."""
    g, op = soft_core_op(8, 0.35, 2.0)
    ev = np.linalg.eigvalsh(ham.dense(op))
    bound = ev[(ev > -C * C) & (ev < 0)]
    gap = np.argmax(np.diff(bound))               # widest spacing between bound states
    # between the midpoint (degenerate fold) and the point where the next
    # state below becomes nearer: the two nearest states straddle the fold
    mid = 0.5 * (bound[gap] + bound[gap + 1])
    sigma = 0.5 * (mid + 0.5 * (bound[gap + 1] + bound[gap - 1]))
    res = lz.lanczos_eigs(op, wl.random_spinor(g, 9), n_want=2, max_iter=256,
                          tol=1e-10, window=None, fold=sigma)
    want = np.sort(ev[np.argsort(np.abs(ev - sigma))[:2]])
    assert want[0] < sigma < want[1]
    norm_a = np.max((ev - sigma) ** 2)
    assert np.allclose(res.values, want, atol=2.2e-16 * norm_a / abs(want[0] - sigma) + 1e-9)


@pytest.mark.parametrize("fold", [None, -1.0])
def test_ritz_vectors_residual_equals_bound(fold):
    g, op = soft_core_op(10, 0.3, 2.0)
    start = wl.positive_energy_packet(g, p0=(0.0, 0.0)) + 1e-3 * wl.random_spinor(g, 4)
    res = lz.lanczos_eigs(op, start, n_want=2, max_iter=200, tol=1e-8,
                          window=(-C * C, 0.0), fold=fold, vectors=True)
    assert len(res.vectors) == res.values.size >= 2
    for lam, y in zip(res.values, res.vectors):
        assert abs(ham.norm(y) - 1.0) <= 1e-12
        r = ham.norm(ham.apply(op, y) - lam * y)
        if fold is None:
            # Ritz pair of A = H - s: the residual is the Eq. 9 bound itself
            j = np.argmin(np.abs(res.all_ritz - lam))
            assert abs(r - res.all_bounds[j]) <= 1e-9 * max(1.0, abs(lam))
        else:
            assert r <= 1e-4


def test_ritz_vector_matches_dense_eigenvector():
    g, op = soft_core_op(8, 0.35, 2.0)
    w, U = np.linalg.eigh(ham.dense(op))
    start = wl.random_spinor(g, 11)
    res = lz.lanczos_eigs(op, start, n_want=1, max_iter=256, tol=1e-11,
                          window=(-C * C, 0.0), vectors=True)
    lam, y = res.values[0], res.vectors[0].reshape(-1)
    j = np.argmin(np.abs(w - lam))
    overlap = abs(np.vdot(U[:, j], y))
    assert abs(lam - w[j]) <= 1e-8
    assert overlap >= 1.0 - 1e-8


def test_breakdown_in_invariant_subspace_gives_exact_energies():
    nx, ny, dx, dy, A = 8, 8, 0.3, 0.3, (1.5, 0.0)
    op = ham.Operator(nx, ny, dx, dy, A=A)
    # three plane-wave eigenvectors (two momenta, both signs of energy at one)
    vecs, energies = [], []
    for jx, jy, sign in ((1, 0, 1), (1, 0, -1), (2, 3, 1)):
        psi, E = plane_wave_eigpair(nx, ny, dx, dy, jx, jy, 2, A, 0.0, sign=sign)
        vecs.append(psi)
        energies.append(E)
    start = vecs[0] + 0.7 * vecs[1] + 0.4 * vecs[2]
    res = lz.lanczos_eigs(op, start, n_want=10, max_iter=50, tol=1e-10,
                          window=(-1e9, 1e9))
    assert res.breakdown and res.iterations == 3
    assert np.allclose(np.sort(res.all_ritz), np.sort(energies), rtol=1e-12, atol=1e-9)
    assert np.allclose(res.values, np.sort(energies), rtol=1e-12, atol=1e-9)


def test_reorthogonalisation_removes_ghost_copies():
    """Loss of orthogonality (Sec. 2): the plain recurrence, run long enough,
    returns converged copies of eigenvalues it already found; with the full
    reorthogonalisation every converged value pairs with its own eigenvalue of
    the dense operator."""
    g = wl.Grid(24, 20, 0.3, 0.3)
    V = wl.soft_core(g, 2.0)
    start = wl.positive_energy_packet(g, p0=(0.0, 0.0)) + 1e-3 * wl.random_spinor(g, 4)
    op = ham.Operator(g.nx, g.ny, g.dx, g.dy, V=V, shift=C * C)
    window = (-C * C, 0.0)
    exact = np.linalg.eigvalsh(ham.dense(op))
    exact = exact[(exact > window[0]) & (exact < window[1])]

    def copies(values):
        # values that share their nearest dense eigenvalue with another value
        nearest = [int(np.argmin(np.abs(exact - v))) for v in values]
        return len(nearest) - len(set(nearest))

    full = lz.lanczos_eigs(op, start, n_want=48, max_iter=400, tol=1e-10, window=window)
    plain = lz.lanczos_eigs(op, start, n_want=48, max_iter=400, tol=1e-10, window=window, reorth=False)
    assert full.values.size >= 8 and copies(full.values) == 0
    assert np.max(np.abs(exact[[int(np.argmin(np.abs(exact - v))) for v in full.values]] - full.values)) < 1e-8
    assert copies(plain.values) >= 1
