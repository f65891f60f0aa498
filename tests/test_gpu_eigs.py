"""Parity of the eigenvalue mode and the Hamiltonian product (CUDA path through
the C ABI) with the CPU FP64 oracle, plus size-independent checks at the full
2048x2048 smoothed-Coulomb workload.

Tolerances: the GPU and the oracle build T_k from the same recurrence but
round differently (sums in another order, alpha accumulated from the two
Gram-Schmidt passes), so T_k agrees to a few ulps of ||A||; a converged Ritz
value is well conditioned and moves by about as much.  Ritz values are
compared to 1e-11 * ||A|| (||A|| <= ~4e4 here); folded mode squares A, so
there the floor is u ||A|| / |lambda - sigma| (the oracle's own pin).
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import lanczos as lz
from paper_1407_7370_gb300 import workloads as wl
from test_oracle_hamiltonian import plane_wave_eigpair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C = 137.036


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_7370_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def make(grid, V=None, A=(0.0, 0.0), shift=0.0, order=2, boundary="periodic", precision="fp64"):
    from paper_1407_7370_gb300 import Propagator
    p = Propagator(grid.nx, grid.ny, grid.dx, grid.dy, order=order, boundary=boundary, m_max=4,
                   precision=precision)
    p.set_fields(None if V is None else torch.from_numpy(np.ascontiguousarray(V)).cuda(), A=A,
                 shift=shift)
    op = ham.Operator(grid.nx, grid.ny, grid.dx, grid.dy, order=order,
                      boundary=ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC,
                      V=V, A=A, shift=shift)
    return p, op


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def norm_a(op):
    """An upper bound of ||H - s|| (Gershgorin on the stencil): the rounding scale."""
    mc2 = op.mass * op.c ** 2
    kin = op.c * (np.sqrt(2.0) * (1.5 if op.order == 4 else 1.0) / min(op.dx, op.dy)
                  + abs(op.A[0]) + abs(op.A[1]))
    v = 0.0 if op.V is None else np.max(np.abs(op.V))
    return mc2 + kin + v + abs(op.shift)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("order,boundary", [(2, "periodic"), (4, "periodic"), (2, "dirichlet"),
                                            (4, "dirichlet")])
def test_apply_hamiltonian_matches_oracle(order, boundary):
    g = wl.Grid(37, 29, 0.11, 0.17)            # ragged against every tile shape
    V = wl.random_potential(g, 3, scale=40.0)
    p, op = make(g, V=V, A=(2.5, -1.25), shift=C * C * 0.5, order=order, boundary=boundary)
    psi = wl.random_spinor(g, 8)
    out = p.apply(dev(psi)).cpu().numpy()
    ref = ham.apply(op, psi)
    assert np.max(np.abs(out - ref)) <= 1e-14 * norm_a(op) * np.max(np.abs(psi))


def soft_core_case(n=24, m=20, dx=0.3, z=2.0):
    g = wl.Grid(n, m, dx, dx)
    V = wl.soft_core(g, z)
    start = wl.positive_energy_packet(g, p0=(0.0, 0.0)) + 1e-3 * wl.random_spinor(g, 4)
    return g, V, start


def test_eigs_direct_matches_oracle_fixed_iterations():
    g, V, start = soft_core_case()
    p, op = make(g, V=V, shift=C * C)
    window = (-C * C, 0.0)
    res = p.eigs(dev(start), n_want=64, max_iter=150, tol=1e-9, window=window, check_every=10)
    ref = lz.lanczos_eigs(op, start, n_want=64, max_iter=150, tol=1e-9, window=window,
                          check_every=10)
    assert res.iterations == ref.iterations == 150
    assert res.values.size == min(64, ref.values.size) and res.values.size >= 2
    scale = 1e-11 * norm_a(op)
    assert np.max(np.abs(res.values - ref.values[: res.values.size])) <= scale
    assert np.all(res.bounds <= 1e-9 * np.maximum(1.0, np.abs(res.values)))
    assert res.n_converged == ref.values.size


def test_eigs_stops_at_the_oracles_iteration():
    g, V, start = soft_core_case(20, 20, 0.3, 3.0)
    p, op = make(g, V=V, shift=C * C)
    window = (-C * C, 0.0)
    for n_want, every in ((1, 5), (3, 7)):
        res = p.eigs(dev(start), n_want=n_want, max_iter=400, tol=1e-10, window=window,
                     check_every=every)
        ref = lz.lanczos_eigs(op, start, n_want=n_want, max_iter=400, tol=1e-10, window=window,
                              check_every=every)
        assert res.iterations == ref.iterations < 400
        assert res.values.size == n_want
        assert np.max(np.abs(res.values - ref.values[:n_want])) <= 1e-11 * norm_a(op)


def test_eigs_without_reorthogonalisation_matches_oracle():
    g, V, start = soft_core_case(16, 18, 0.3, 2.0)
    p, op = make(g, V=V, shift=C * C)
    window = (-C * C, 0.0)
    res = p.eigs(dev(start), n_want=64, max_iter=150, tol=1e-8, window=window, reorth=False)
    ref = lz.lanczos_eigs(op, start, n_want=64, max_iter=150, tol=1e-8, window=window,
                          reorth=False)
    assert res.iterations == ref.iterations == 150
    assert res.values.size >= 1 and ref.values.size >= 1
    # without reorthogonalisation rounding differences grow once values
    # converge (Sec. 2), so compare the converged values as sets
    for v in res.values:
        assert np.min(np.abs(ref.values - v)) <= 1e-10 * norm_a(op)
    for v in ref.values:
        assert np.min(np.abs(res.values - v)) <= 1e-10 * norm_a(op)


def test_eigs_folded_matches_oracle():
    g = wl.Grid(10, 10, 0.3, 0.3)
    V = wl.soft_core(g, 3.0)
    p, op = make(g, V=V, shift=C * C)
    start = wl.random_spinor(g, 5)
    sigma = -2.0
    res = p.eigs(dev(start), n_want=3, max_iter=200, tol=1e-9, fold=sigma, vectors=True)
    ref = lz.lanczos_eigs(op, start, n_want=3, max_iter=200, tol=1e-9, window=None, fold=sigma,
                          vectors=True)
    ev = np.linalg.eigvalsh(ham.dense(op))
    want = np.sort(ev[np.argsort(np.abs(ev - sigma))[:3]])
    assert res.iterations == ref.iterations
    assert res.values.size == 3
    floor = 2.2e-16 * norm_a(op) ** 2 / np.abs(want - sigma)
    assert np.all(np.abs(res.values - ref.values) <= 2 * floor)
    assert np.all(np.abs(res.values - want) <= res.bounds + floor)
    # a Ritz vector of A = (H - s - sigma)^2 is fixed to an angle of about
    # u ||A|| / gap, gap its distance to the rest of A's spectrum
    mu = (ev - sigma) ** 2
    for lam, y, yr in zip(res.values, res.vectors.cpu().numpy(), ref.vectors):
        th = (lam - sigma) ** 2
        gap = np.sort(np.abs(mu - th))[1]
        angle = 4 * 2.2e-16 * norm_a(op) ** 2 / gap
        assert abs(abs(np.vdot(yr.reshape(-1), y.reshape(-1))) - 1.0) <= 0.5 * angle ** 2 + 1e-12


def test_ritz_vectors_match_oracle_and_residual_identity():
    g, V, start = soft_core_case(20, 16, 0.3, 2.0)
    p, op = make(g, V=V, shift=C * C)
    window = (-C * C, 0.0)
    res = p.eigs(dev(start), n_want=3, max_iter=200, tol=1e-10, window=window, vectors=True)
    ref = lz.lanczos_eigs(op, start, n_want=3, max_iter=200, tol=1e-10, window=window,
                          vectors=True)
    assert res.iterations == ref.iterations
    ys = res.vectors
    for l in range(res.values.size):
        y = ys[l]
        assert abs(torch.linalg.vector_norm(y).item() - 1.0) <= 1e-12
        # Eq. 10: ||A y - theta y|| = |beta_k t_k| for a Ritz pair
        r = torch.linalg.vector_norm(p.apply(y) - res.values[l] * y).item()
        assert r <= res.bounds[l] + 1e-10 * norm_a(op)
        yr = ref.vectors[l].reshape(-1)
        gap = np.min(np.abs(np.delete(ref.all_ritz, np.argmin(np.abs(ref.all_ritz - ref.values[l])))
                            - ref.values[l]))
        if gap > 1e-6:   # non-degenerate: the vector is unique up to a phase
            assert abs(abs(np.vdot(yr, y.cpu().numpy().reshape(-1))) - 1.0) <= 1e-8


def test_eigs_breakdown_gives_exact_free_energies():
    nx, ny, dx, dy, A = 8, 8, 0.3, 0.3, (1.5, 0.0)
    g = wl.Grid(nx, ny, dx, dy)
    p, op = make(g, A=A)
    vecs, energies = [], []
    for jx, jy, sign in ((1, 0, 1), (1, 0, -1), (2, 3, 1)):
        psi, E = plane_wave_eigpair(nx, ny, dx, dy, jx, jy, 2, A, 0.0, sign=sign)
        vecs.append(psi)
        energies.append(E)
    start = vecs[0] + 0.7 * vecs[1] + 0.4 * vecs[2]
    res = p.eigs(dev(start), n_want=10, max_iter=50, tol=1e-10, window=(-1e9, 1e9))
    assert res.breakdown and res.iterations == 3
    assert np.allclose(res.values, np.sort(energies), rtol=1e-12, atol=0)


def test_eigs_rejects_bad_arguments():
    from paper_1407_7370_gb300._native import DiracError
    g, V, start = soft_core_case(8, 8, 0.3, 2.0)
    p, _ = make(g, V=V, shift=C * C)
    s = dev(start)
    with pytest.raises(DiracError):
        p.eigs(s, n_want=0, max_iter=10, tol=1e-8, window=(-1.0, 0.0))
    with pytest.raises(DiracError):
        p.eigs(s, n_want=1, max_iter=10, tol=1e-8, window=(0.0, -1.0))
    with pytest.raises(DiracError):
        p.eigs(torch.zeros_like(s), n_want=1, max_iter=10, tol=1e-8, window=(-1.0, 0.0))


@pytest.mark.slow
def test_eigs_48_grid_matches_dense_eigh():
    """Smoothed Coulomb Z = 20, a = 0.5 on a 48x48 grid, dx = 0.1: the eigen
    mode's converged values against the dense spectrum of the same operator."""
    import scipy.linalg
    g = wl.Grid(48, 48, 0.1, 0.1)
    V = wl.smoothed_coulomb(g, 20.0, 0.5)
    p, op = make(g, V=V, shift=C * C)
    x, y = g.coords()
    start = np.zeros((48, 48, 2), complex)
    start[..., 0] = np.exp(-(x * x + y * y) * 4.0)
    start = start + 1e-3 * wl.random_spinor(g, 1)
    window = (-C * C, 0.0)
    res = p.eigs(dev(start), n_want=8, max_iter=600, tol=1e-9, window=window, check_every=10)
    ev = scipy.linalg.eigh(ham.dense(op), eigvals_only=True, subset_by_value=window)
    assert res.values.size >= 4
    for v, b in zip(res.values, res.bounds):
        assert np.min(np.abs(ev - v)) <= b + 1e-11 * norm_a(op)
    # the lowest bound state is found
    assert abs(res.values[0] - ev[0]) <= 1e-8 * abs(ev[0])


@pytest.mark.slow
@pytest.mark.parametrize("z,min_found", [(1.0, 0), (20.0, 1), (60.0, 2)])
def test_eigs_full_size_coulomb_2048(z, min_found):
    """2048x2048, dx = 0.02, V = -Z/sqrt(r^2 + 0.25), up to 400 iterations: the
    converged Ritz pairs satisfy the Eq. 10 residual identity with the GPU
    Hamiltonian, lie in the window, and are orthonormal.

    How many converge in 400 iterations depends on Z.  With central
    differences the kinetic term tops out at c sqrt(2)/dx ~ 9700, so the
    positive band runs from m c^2 to about m c^2 + 2350, and the negative band
    lies 2 m c^2 ~ 37600 below it: the bound states sit at the inner edge of a
    spectrum about 42000 wide, and the Krylov space resolves the deepest of
    them first.  Measured: Z = 1 (binding of order 1 hartree) converges none
    in 400 iterations, Z = 20 one (about -29.8), Z = 60 two or three.
    """
    n = 2048
    g = wl.Grid(n, n, 0.02, 0.02)
    V = wl.smoothed_coulomb(g, z, 0.5)
    p, op = make(g, V=V, shift=C * C)
    x, y = g.coords()
    start = np.zeros((n, n, 2), complex)
    start[..., 0] = np.exp(-(x * x + y * y) * z)
    start = start + 1e-3 * wl.random_spinor(g, 2) * np.exp(-(x * x + y * y))[..., None]
    res = p.eigs(dev(start), n_want=8, max_iter=400, tol=1e-8, window=(-C * C, 0.0),
                 vectors=True)
    assert res.iterations <= 400
    assert res.values.size >= min_found
    assert res.n_converged >= res.values.size
    # the well binds: T_k has Ritz values below m c^2 even where none has
    # converged yet (measured: 2 for Z = 1, 11 for Z = 20, 21 for Z = 60)
    assert res.n_in_window >= 1
    if res.values.size == 0:
        return
    Y = res.vectors.reshape(res.values.size, -1)
    gram = (Y.conj() @ Y.T).cpu().numpy()
    assert np.max(np.abs(gram - np.eye(res.values.size))) <= 1e-8
    for l in range(res.values.size):
        yl = res.vectors[l]
        r = torch.linalg.vector_norm(p.apply(yl) - res.values[l] * yl).item()
        assert r <= res.bounds[l] * (1 + 1e-6) + 1e-10 * norm_a(op)
        assert -C * C < res.values[l] < 0.0
    # the ground state sits below the top of the smoothed well's depth
    assert res.values[0] > -z / 0.5 - 1e-6


def test_eigs_launch_count_and_kernel_timing():
    g, V, start = soft_core_case(16, 16, 0.3, 2.0)
    p, _ = make(g, V=V, shift=C * C)
    p.profile(True)
    res = p.eigs(dev(start), n_want=200, max_iter=30, tol=1e-14, window=(-C * C, 0.0),
                 check_every=10)
    p.profile(False)
    assert res.iterations == 30
    # start vector + 30 x (product + 2 x (inner products, sums, update)) + 3 checks x 3
    assert res.launches == 1 + 30 * 7 + 3 * 3
    assert res.ms["apply"] > 0 and res.ms["dot"] > 0 and res.ms["update"] > 0 and res.ms["other"] > 0


def test_eigs_mixed_stencil_close_to_fp64():
    """FP32 off-diagonal stencil products (FP64 diagonal, FP64
    reorthogonalisation and Ritz values): each product carries a rounding
    error of a few u32 times ||K|| ||q||, K = c sigma.(p + A) the part done in
    FP32, so the Ritz values move by at most that much, plus the looser
    convergence tolerance.  The grid is small enough for the whole spectrum
    of the discrete operator (dense matrix, LAPACK), which has a close
    quadruplet near -2.03 au: the looser tolerance admits the inner pair."""
    g, V, start = soft_core_case(24, 20, 0.3, 2.0)
    window = (-C * C, 0.0)
    p64, op = make(g, V=V, shift=C * C)
    p32, _ = make(g, V=V, shift=C * C, precision="mixed")
    r64 = p64.eigs(dev(start), n_want=64, max_iter=150, tol=1e-9, window=window)
    r32 = p32.eigs(dev(start), n_want=64, max_iter=150, tol=1e-6, window=window)
    assert r32.values.size >= 2
    exact = np.linalg.eigvalsh(ham.dense(op))
    exact = exact[(exact > window[0]) & (exact < window[1])]
    kin = op.c * (np.sqrt(2.0) / min(op.dx, op.dy) + abs(op.A[0]) + abs(op.A[1]))
    for v, b in zip(r32.values, r32.bounds):
        assert np.min(np.abs(exact - v)) <= 4 * 2.0 ** -24 * kin + 2 * b, (v, b)
    assert r64.values.size >= 2
    for v in r64.values:
        assert np.min(np.abs(exact - v)) <= 1e-11 * norm_a(op)


def test_full_reorthogonalisation_has_no_ghost_eigenvalues():
    """Without reorthogonalisation the Lanczos recurrence loses orthogonality
    and converged Ritz values reappear as spurious copies (Sec. 2).  With the
    full (twice applied) Gram-Schmidt every converged Ritz value must pair with
    its own eigenvalue of the dense discrete operator -- including inside the
    near-degenerate quadruplet near -2.03 au (spacings down to 6e-5) -- so a
    ghost copy has no partner left within the rounding scale."""
    g, V, start = soft_core_case(24, 20, 0.3, 2.0)
    window = (-C * C, 0.0)
    p, op = make(g, V=V, shift=C * C)
    res = p.eigs(dev(start), n_want=48, max_iter=400, tol=1e-10, window=window)
    exact = np.linalg.eigvalsh(ham.dense(op))
    exact = exact[(exact > window[0]) & (exact < window[1])]
    assert res.values.size >= 8
    tol = 1e-11 * norm_a(op) + 2 * np.max(res.bounds)
    assert tol < 6e-5
    used = set()
    for v in np.sort(res.values):
        free_idx = [j for j in range(exact.size) if j not in used]
        j = min(free_idx, key=lambda k: abs(exact[k] - v))
        assert abs(exact[j] - v) <= tol, (v, exact[j])
        used.add(j)


@pytest.mark.parametrize("order,boundary", [(4, "dirichlet"), (4, "periodic"), (2, "dirichlet")])
def test_eigs_other_stencils_and_a_field_match_oracle(order, boundary):
    """The eigen mode with the fourth-order stencil, Dirichlet boundaries and
    a uniform vector potential (both components): Ritz values, iteration
    count and convergence as the oracle."""
    g, V, start = soft_core_case(22, 18, 0.3, 2.0)
    A = (5.0, -2.0)
    p, op = make(g, V=V, A=A, shift=C * C, order=order, boundary=boundary)
    window = (-C * C, 0.0)
    res = p.eigs(dev(start), n_want=8, max_iter=400, tol=1e-9, window=window, check_every=10)
    ref = lz.lanczos_eigs(op, start, n_want=8, max_iter=400, tol=1e-9, window=window, check_every=10)
    assert res.iterations == ref.iterations
    assert res.values.size == ref.values.size >= 2
    assert np.max(np.abs(res.values - ref.values)) <= 1e-11 * norm_a(op)
