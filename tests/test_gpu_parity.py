"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerance (FP64 path): relative L2 of psi at most 1e-10 per unit of simulated
time, the propagation target of this library, with a floor of 1e-14 per step
for runs too short for that to exceed rounding (both sides round differently:
the GPU sums in a different order and evaluates exp(-iT dt) e_1 by a
Chebyshev expansion where the oracle diagonalises T).
"""
import ctypes

import numpy as np
import pytest

from oracle import free
from oracle import hamiltonian as ham
from oracle import lanczos as lz
from paper_1407_7370_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C = 137.036


def fp64_tol(steps, dt):
    return max(1e-10 * steps * dt, 1e-14 * steps)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_7370_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def gpu_run(grid, psi0, dt, m, steps, V=None, A=(0.0, 0.0), order=2, boundary="periodic",
            shift=0.0, tol=0.0, A_steps=None, info=True, precision="fp64", step_mode="auto"):
    from paper_1407_7370_gb300 import Propagator
    prop = Propagator(grid.nx, grid.ny, grid.dx, grid.dy, order=order, boundary=boundary, m_max=m,
                      precision=precision)
    prop.set_step_mode(step_mode)
    prop.set_fields(None if V is None else torch.from_numpy(V).cuda(), A=A, shift=shift)
    psi = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    inf = prop.steps(psi, steps, dt, m, tol=tol, A=A_steps, info=info)
    return psi.cpu().numpy(), inf, prop


def oracle_op(grid, V=None, A=(0.0, 0.0), order=2, boundary=ham.PERIODIC, shift=0.0):
    return ham.Operator(grid.nx, grid.ny, grid.dx, grid.dy, order=order, boundary=boundary,
                        V=V, A=A, shift=shift)


# ---------------------------------------------------------------------------
def test_device_small_exponential_matches_scipy():
    import scipy.linalg
    from paper_1407_7370_gb300 import tridiag_expm_device
    rng = np.random.default_rng(0)
    for k in (1, 2, 5, 10, 20, 32):
        for R in (0.05, 2.0, 10.0, 40.0):
            alpha = rng.uniform(-1, 1, k)
            beta = np.abs(rng.uniform(0.1, 0.5, max(k - 1, 0)))
            T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
            ev = np.linalg.eigvalsh(T)
            lo, hi = ev[0] - 0.1, ev[-1] + 0.1
            dt = R / (0.5 * (hi - lo))
            ref = scipy.linalg.expm(-1j * dt * T)[:, 0]
            v = tridiag_expm_device(alpha, beta, dt, lo, hi)
            assert np.max(np.abs(v - ref)) <= 2e-14 * (1 + R), (k, R)


def test_free_packet_64_full_run_matches_oracle():
    """64x64, dx=0.1, m=10, dt=1e-4, 100 steps: the oracle-sized propagation case."""
    cfg = wl.FREE_PACKET_64
    g = cfg["grid"]
    psi0 = wl.positive_energy_packet(g, p0=cfg["p0"], sigma_x=cfg["sigma_x"])
    out, info, _ = gpu_run(g, psi0, cfg["dt"], cfg["m"], cfg["steps"])
    ref, infos = lz.propagate(oracle_op(g), psi0.copy(), cfg["dt"], cfg["m"], cfg["steps"])
    err = lz.rel_l2(out, ref)
    assert err <= 1e-10 * cfg["steps"] * cfg["dt"], err
    # both against the closed-form free propagation, within the cumulative bound (Sec. 6)
    exact = free.propagate(oracle_op(g), psi0.copy(), cfg["dt"], cfg["steps"])
    cum = sum(i.err_est for i in infos)
    assert ham.norm(out - exact) <= cum + 1e-12 * ham.norm(exact)
    # estimates below ~1e-14 ||psi|| are rounding noise on both sides
    assert abs(info.cum_err - cum) <= 1e-6 * cum + 1e-14 * ham.norm(psi0) * cfg["steps"]


def test_step_scalars_match_oracle():
    g = wl.Grid(64, 48, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 5.0))
    V = wl.smoothed_coulomb(g, 3.0, 0.5)
    dt, m = 1e-4, 12
    out, info, _ = gpu_run(g, psi0, dt, m, 1, V=V, A=(4.0, -2.0))
    ref, oi = lz.krylov_step(oracle_op(g, V=V, A=(4.0, -2.0)), psi0.copy(), dt, m)
    assert info.k_used == oi.k_used == m
    assert np.allclose(info.alpha, oi.alpha / dt, rtol=1e-12, atol=1e-10)
    assert np.allclose(info.beta[: m - 1], oi.beta[: m - 1] / dt, rtol=1e-9, atol=1e-9)
    assert abs(info.beta[m - 1] - oi.beta[m - 1] / dt) <= 1e-6 * oi.beta[m - 1] / dt
    assert abs(info.err_est - oi.err_est) <= 1e-6 * oi.err_est + 1e-14 * oi.norm
    assert abs(info.energy - oi.energy) <= 1e-12 * abs(oi.energy)
    assert abs(info.norm - oi.norm) <= 1e-13 * oi.norm
    assert lz.rel_l2(out, ref) <= fp64_tol(1, dt)


def test_error_estimate_matches_oracle_when_it_is_large():
    g = wl.Grid(64, 64, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 0.0)) + 0.05 * wl.random_spinor(g, 3)
    for m in (2, 3, 4):
        out, info, _ = gpu_run(g, psi0, 1e-4, m, 1)
        ref, oi = lz.krylov_step(oracle_op(g), psi0.copy(), 1e-4, m)
        assert oi.err_est > 1e-10 * oi.norm
        assert abs(info.err_est - oi.err_est) <= 1e-6 * oi.err_est
        assert lz.rel_l2(out, ref) <= 1e-12


CASES = [
    # nx, ny, order, boundary, V, A
    (37, 23, 2, "periodic", True, (3.0, -1.5)),
    (33, 9, 4, "periodic", True, (0.0, 2.0)),
    (40, 17, 2, "dirichlet", True, (1.0, 1.0)),
    (35, 11, 4, "dirichlet", False, (2.5, 0.0)),
    (3, 5, 2, "periodic", True, (1.0, 0.5)),
    (7, 1, 2, "periodic", False, (1.0, 0.0)),
    (1, 9, 4, "dirichlet", True, (0.0, 0.3)),
    (64, 8, 2, "periodic", False, (0.0, 0.0)),
]


@pytest.mark.parametrize("nx,ny,order,boundary,hasv,A", CASES)
def test_ragged_small_and_boundary_grids(nx, ny, order, boundary, hasv, A):
    g = wl.Grid(nx, ny, 0.1, 0.13)
    psi0 = wl.random_spinor(g, nx * 100 + ny) * 0.1
    V = wl.random_potential(g, 7, scale=20.0) if hasv else None
    dt, m, steps = 1e-4, 6, 3
    b = ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC
    out, info, _ = gpu_run(g, psi0, dt, m, steps, V=V, A=A, order=order, boundary=boundary)
    ref, oinf = lz.propagate(oracle_op(g, V=V, A=A, order=order, boundary=b), psi0.copy(), dt, m, steps)
    assert info.k_used == oinf[-1].k_used
    assert lz.rel_l2(out, ref) <= fp64_tol(steps, dt)


def test_tolerance_mode_matches_oracle_k():
    g = wl.Grid(48, 48, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    dt, m = 1e-4, 20
    for tol in (1e-7, 1e-10):
        out, info, _ = gpu_run(g, psi0, dt, m, 1, tol=tol)
        ref, oi = lz.krylov_step(oracle_op(g), psi0.copy(), dt, m, tol=tol)
        assert info.k_used == oi.k_used < m
        assert lz.rel_l2(out, ref) <= fp64_tol(1, dt)


def test_breakdown_on_plane_wave_eigenvector():
    from tests.test_oracle_hamiltonian import plane_wave_eigpair
    g = wl.Grid(16, 16, 0.1, 0.1)
    psi, E = plane_wave_eigpair(16, 16, 0.1, 0.1, 3, 1, 2, (2.0, 0.0), 0.0)
    out, info, _ = gpu_run(g, psi, 1e-4, 10, 1, A=(2.0, 0.0))
    assert info.k_used == 1 and info.breakdown
    assert np.max(np.abs(out - np.exp(-1j * E * 1e-4) * psi)) <= 1e-13


def test_energy_shift_does_not_change_the_step():
    g = wl.Grid(32, 32, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    a, _, _ = gpu_run(g, psi0, 1e-4, 10, 5)
    b, _, _ = gpu_run(g, psi0, 1e-4, 10, 5, shift=C * C)
    assert lz.rel_l2(b, a) <= fp64_tol(5, 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bitwise_deterministic(precision):
    g = wl.Grid(96, 80, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    V = wl.smoothed_coulomb(g, 2.0, 0.5)
    shift = C * C if precision == "mixed" else 0.0
    a, ia, _ = gpu_run(g, psi0, 1e-4, 10, 4, V=V, precision=precision, shift=shift)
    b, ib, _ = gpu_run(g, psi0, 1e-4, 10, 4, V=V, precision=precision, shift=shift)
    assert np.array_equal(a, b) and ia.err_est == ib.err_est


@pytest.mark.parametrize("nx,ny", [(64, 64), (70, 64), (64, 44), (70, 44), (33, 17), (130, 47), (56, 16),
                                   (57, 17)])
@pytest.mark.parametrize("boundary", ["periodic", "dirichlet"])
def test_mixed_one_launch_tile_shapes(nx, ny, boundary):
    """The mixed one-launch step on grids whose tiles (32 x 16) are whole,
    ragged in x, in y, or in both, against the oracle: every tile, however
    its stage is filled (tensor copies with halo patches, or row copies),
    gives the same product."""
    g = wl.Grid(nx, ny, 0.1, 0.1)
    psi0 = 0.1 * wl.random_spinor(g, nx + 7 * ny)
    b = ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC
    out, _, _ = gpu_run(g, psi0, 1e-5, 8, 2, A=(1.0, 0.5), boundary=boundary, precision="mixed",
                        step_mode="one_launch")
    ref, _ = lz.propagate(oracle_op(g, A=(1.0, 0.5), boundary=b), psi0.copy(), 1e-5, 8, 2)
    assert lz.rel_l2(out, ref) <= mixed_tol(2, 1e-5, hnorm(g, (1.0, 0.5)))


def test_nonfinite_input_is_reported_and_psi_kept():
    from paper_1407_7370_gb300 import Propagator
    from paper_1407_7370_gb300._native import DiracError, ENONFINITE
    g = wl.Grid(32, 16, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g)
    psi0[3, 4, 1] = np.nan
    prop = Propagator(32, 16, 0.1, 0.1, m_max=8)
    prop.set_fields()
    psi = torch.from_numpy(psi0.copy()).cuda()
    with pytest.raises(DiracError) as e:
        prop.step(psi, 1e-4, 8, info=True)
    assert e.value.status == ENONFINITE
    back = psi.cpu().numpy()
    assert np.array_equal(np.isnan(back), np.isnan(psi0))
    assert np.array_equal(np.nan_to_num(back), np.nan_to_num(psi0))
    # the context stays usable
    psi.copy_(torch.from_numpy(wl.positive_energy_packet(g)))
    info = prop.step(psi, 1e-4, 8, info=True)
    assert info.k_used == 8


def test_invalid_arguments_are_rejected():
    from paper_1407_7370_gb300 import Propagator
    from paper_1407_7370_gb300 import _native as nat
    g = wl.Grid(16, 16, 0.1, 0.1)
    prop = Propagator(16, 16, 0.1, 0.1, m_max=8)
    psi = torch.from_numpy(wl.positive_energy_packet(g)).cuda()
    L = nat.lib()
    p = ctypes.c_void_p(psi.data_ptr())
    assert L.dirac_lanczos_step(prop._ctx, p, 1e-4, 8, 0.0, None) == nat.ESTATE
    prop.set_fields()
    assert L.dirac_lanczos_step(prop._ctx, p, 1e-4, 9, 0.0, None) == nat.EINVAL
    assert L.dirac_lanczos_step(prop._ctx, p, 1e-4, 0, 0.0, None) == nat.EINVAL
    assert L.dirac_lanczos_step(prop._ctx, p, 0.0, 8, 0.0, None) == nat.EINVAL
    assert L.dirac_lanczos_step(prop._ctx, p, 1e-4, 8, -1.0, None) == nat.EINVAL
    assert L.dirac_lanczos_step(prop._ctx, ctypes.c_void_p(psi.data_ptr() + 16), 1e-4, 8, 0.0,
                                None) == nat.EINVAL
    assert L.dirac_lanczos_step(prop._ctx, p, 1.0, 8, 0.0, None) == nat.EINVAL   # dt*||H|| > 90
    assert L.dirac_sync(prop._ctx) == nat.OK


def test_host_buffer_call_equals_device_call():
    from paper_1407_7370_gb300 import Propagator
    g = wl.Grid(64, 64, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 0.0))
    A = np.stack([np.linspace(0, 5, 6), np.zeros(6)], axis=1)
    dev, _, _ = gpu_run(g, psi0, 1e-4, 10, 6, A_steps=A)
    prop = Propagator(64, 64, 0.1, 0.1, m_max=10)
    prop.set_fields()
    host = torch.from_numpy(psi0.copy()).pin_memory()
    prop.propagate_host(host, 6, 1e-4, 10, A=A)
    assert np.array_equal(host.numpy(), dev)


@pytest.mark.parametrize("precision,mode,per_step", [
    ("fp64", "passes", 7 + 2 + 1),      # m passes + 2 spare launches for re-runs + recombine
    ("fp64", "one_launch", 1),
    ("fp64", "auto", 1),
    ("mixed", "passes", 7 + 3 + 1),     # the mixed path keeps 2 + m / 5 spare launches
    ("mixed", "auto", 7 + 3 + 1),
    ("mixed", "one_launch", 1)])
def test_kernel_launch_count(precision, mode, per_step):
    g = wl.Grid(32, 32, 0.1, 0.1)
    _, _, prop = gpu_run(g, wl.positive_energy_packet(g), 1e-4, 7, 3, precision=precision,
                         step_mode=mode)
    assert prop.kernel_launches == 1 + 3 * per_step     # the probe, then the steps


@pytest.mark.parametrize("precision,mode", [("fp64", "one_launch"), ("fp64", "passes"),
                                            ("mixed", "passes"), ("mixed", "one_launch")])
@pytest.mark.parametrize("m", [1, 2, 3, 32])
def test_krylov_dimension_extremes(precision, mode, m):
    """m = 1 (psi' = exp(-i alpha_1 dt) psi), m = 2 and the largest Krylov
    dimension the device recurrence holds (32, one warp), against the oracle."""
    g = wl.Grid(40, 36, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(6.0, 2.0)) + 0.02 * wl.random_spinor(g, 5)
    V = wl.soft_core(g, 1.5)
    shift = C * C if precision == "mixed" else 0.0
    dt = 2e-4 if m > 2 else 2e-6
    out, info, _ = gpu_run(g, psi0, dt, m, 3, V=V, A=(3.0, -1.0), shift=shift, precision=precision,
                           step_mode=mode)
    op = oracle_op(g, V=V, A=(3.0, -1.0), shift=shift)
    ref = psi0.copy()
    for _ in range(3):
        ref, oi = lz.krylov_step(op, ref, dt, m)
    assert info.k_used == oi.k_used == m
    tol = fp64_tol(3, dt) if precision == "fp64" else mixed_tol(3, dt, hnorm(g, (3.0, -1.0), V))
    assert lz.rel_l2(out, ref) <= tol


@pytest.mark.parametrize("precision,mode", [("fp64", "one_launch"), ("fp64", "passes"),
                                            ("mixed", "passes"), ("mixed", "one_launch")])
def test_zero_state_stays_zero(precision, mode):
    """exp(-i H dt) 0 = 0: a zero state is a valid input, not an error."""
    g = wl.Grid(33, 20, 0.1, 0.1)
    psi0 = np.zeros((g.ny, g.nx, 2), complex)
    out, info, prop = gpu_run(g, psi0, 1e-4, 8, 3, A=(1.0, 0.5), precision=precision, step_mode=mode)
    assert not np.any(out)
    assert info.norm == 0.0 and info.k_used == 1 and info.err_est == 0.0
    # and the context goes on with a real state
    psi1 = wl.positive_energy_packet(g, p0=(3.0, 0.0))
    psi = torch.from_numpy(psi1.copy()).cuda()
    prop.steps(psi, 2, 1e-4, 8)
    ref, _, _ = gpu_run(g, psi1, 1e-4, 8, 2, A=(1.0, 0.5), precision=precision, step_mode=mode)
    # the first real step starts from the zero state's stencil shift and
    # re-runs its first pass with the Rayleigh quotient: same T to rounding
    tol = 1e-12 if precision == "fp64" else mixed_tol(2, 1e-4, hnorm(g, (1.0, 0.5)))
    assert lz.rel_l2(psi.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("mode", ["one_launch", "passes"])
def test_pass_rerun_after_a_far_stencil_shift(mode):
    """A step of the zero state leaves the first stencil shift at 0; the next
    state is a plane-wave eigenvector plus 1e-7 noise, so ||y^||^2 / s2 of its
    first pass is ~1e13 (beyond the FP64 limit of 1e12): the device re-runs
    the pass with sigma = alpha_1 and the step still matches the oracle."""
    from paper_1407_7370_gb300 import Propagator
    from tests.test_oracle_hamiltonian import plane_wave_eigpair
    g = wl.Grid(32, 24, 0.1, 0.1)
    pw, _ = plane_wave_eigpair(g.nx, g.ny, g.dx, g.dy, 2, 1, 2, (0.0, 0.0), 0.0)
    psi1 = pw + 1e-7 * wl.random_spinor(g, 21)
    prop = Propagator(g.nx, g.ny, g.dx, g.dy, m_max=8)
    prop.set_step_mode(mode)
    prop.set_fields()
    zero = torch.zeros((g.ny, g.nx, 2), dtype=torch.complex128, device="cuda")
    prop.steps(zero, 1, 1e-4, 8)
    psi = torch.from_numpy(psi1.copy()).cuda()
    info = prop.steps(psi, 1, 1e-4, 8, info=True)
    assert info.kappa_max > 1e12          # the pass was re-run
    ref, _ = lz.krylov_step(oracle_op(g), psi1.copy(), 1e-4, 8)
    assert lz.rel_l2(psi.cpu().numpy(), ref) <= fp64_tol(1, 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_is_bitwise(precision):
    """psi and the exported scalar block taken between steps let a new
    context continue bitwise as the original does, cumulative estimate
    included."""
    from paper_1407_7370_gb300 import Propagator
    g = wl.Grid(70, 44, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(8.0, -3.0))
    V = wl.soft_core(g, 2.0)
    rng = np.random.default_rng(4)
    A = rng.uniform(-10, 10, size=(6, 2))
    shift = C * C if precision == "mixed" else 0.0

    def fresh():
        p = Propagator(g.nx, g.ny, g.dx, g.dy, m_max=12, precision=precision)
        p.set_fields(torch.from_numpy(V).cuda(), shift=shift)
        return p

    a = fresh()
    psi = torch.from_numpy(psi0.copy()).cuda()
    a.steps(psi, 3, 1e-4, 12, A=A[:3])
    state, ck = a.export_state(), psi.clone()
    ia = a.steps(psi, 3, 1e-4, 12, A=A[3:], info=True)
    b = fresh()
    b.import_state(state)
    ib = b.steps(ck, 3, 1e-4, 12, A=A[3:], info=True)
    assert torch.equal(ck, psi)
    assert ib.cum_err == ia.cum_err and ib.k_used == ia.k_used


@pytest.mark.parametrize("nx,ny", [(1, 37), (29, 1), (2, 2), (3, 5)])
@pytest.mark.parametrize("order,boundary", [(2, "periodic"), (4, "dirichlet")])
def test_degenerate_thin_grids(nx, ny, order, boundary):
    """One-site-wide, two-by-two and three-by-five grids: the stencil wraps
    onto itself (periodic) or sees only zeros (Dirichlet); both launch forms
    against the oracle."""
    g = wl.Grid(nx, ny, 0.1, 0.1)
    psi0 = wl.random_spinor(g, 13)
    b = ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC
    m = min(6, 2 * nx * ny)
    op = oracle_op(g, A=(2.0, -1.0), order=order, boundary=b)
    ref = psi0.copy()
    for _ in range(3):
        ref, oi = lz.krylov_step(op, ref, 1e-3, m)
    for mode in ("one_launch", "passes"):
        out, info, _ = gpu_run(g, psi0, 1e-3, m, 3, A=(2.0, -1.0), order=order, boundary=boundary,
                               step_mode=mode)
        assert info.k_used == oi.k_used
        assert lz.rel_l2(out, ref) <= fp64_tol(3, 1e-3)


@pytest.mark.parametrize("precision,mode", [("fp64", "one_launch"), ("fp64", "passes"),
                                            ("mixed", "passes")])
def test_backward_steps(precision, mode):
    """dt < 0: psi <- exp(+i H |dt|) psi, against the oracle (the dense
    exponential pins the oracle's backward step); a forward run followed by
    the backward run with the fields in reverse order returns to psi_0."""
    g = wl.Grid(40, 32, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(6.0, 2.0))
    V = wl.soft_core(g, 1.0)
    rng = np.random.default_rng(8)
    A = rng.uniform(-5, 5, size=(4, 2))
    shift = C * C if precision == "mixed" else 0.0
    back, _, _ = gpu_run(g, psi0, -1e-4, 12, 4, V=V, A_steps=A, precision=precision, step_mode=mode,
                         shift=shift)
    op = oracle_op(g, V=V, shift=shift)
    ref = psi0.copy()
    for s in range(4):
        op.A = tuple(A[s])
        ref, _ = lz.krylov_step(op, ref, -1e-4, 12)
    hn = max(hnorm(g, tuple(a), V) for a in A)
    tol = fp64_tol(4, 1e-4) if precision == "fp64" else mixed_tol(4, 1e-4, hn)
    assert lz.rel_l2(back, ref) <= tol
    fwd, _, _ = gpu_run(g, psi0, 1e-4, 12, 4, V=V, A_steps=A, precision=precision, step_mode=mode,
                        shift=shift)
    ret, _, _ = gpu_run(g, fwd, -1e-4, 12, 4, V=V, A_steps=A[::-1].copy(), precision=precision,
                        step_mode=mode, shift=shift)
    assert lz.rel_l2(ret, psi0) <= 2 * tol


def test_one_launch_barrier_timeout_is_reported_and_the_context_recovers():
    """Every grid-barrier wait of the one-launch step is bounded: a step whose
    barriers wait for one CTA more than the launch has ends with DIRAC_ECUDA
    after about a second, psi untouched, and the next steps are correct."""
    from paper_1407_7370_gb300 import Propagator
    from paper_1407_7370_gb300 import _native as nat
    g = wl.Grid(64, 48, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(4.0, 1.0))
    prop = Propagator(g.nx, g.ny, g.dx, g.dy, m_max=10)
    prop.set_fields()
    psi = torch.from_numpy(psi0.copy()).cuda()
    st = nat.lib().dirac_debug_barrier_timeout(prop._ctx, ctypes.c_void_p(psi.data_ptr()), 1e-4, 10)
    assert st == nat.ECUDA
    assert b"barrier" in nat.lib().dirac_last_error()
    assert np.array_equal(psi.cpu().numpy(), psi0)
    prop.steps(psi, 3, 1e-4, 10)
    ref, _, _ = gpu_run(g, psi0, 1e-4, 10, 3)
    assert lz.rel_l2(psi.cpu().numpy(), ref) <= 1e-14


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny,order,boundary,hasv,tol", [(45, 37, 2, "periodic", True, 0.0),
                                                           (70, 33, 4, "dirichlet", False, 0.0),
                                                           (96, 64, 2, "periodic", False, 1e-9)])
def test_one_launch_step_agrees_with_per_pass_launches(precision, nx, ny, order, boundary, hasv, tol):
    """The cooperative one-launch step and the per-pass launches compute the
    same recurrence; only the order in which CTA partials are added differs."""
    g = wl.Grid(nx, ny, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(3.0, -2.0)) + 0.05 * wl.random_spinor(g, 9)
    V = wl.soft_core(g, 1.0) if hasv else None
    rng = np.random.default_rng(3)
    A = rng.uniform(-5, 5, size=(6, 2))
    shift = 137.036 ** 2 if precision == "mixed" else 0.0
    outs = {}
    modes = ("passes", "one_launch")
    for mode in modes:
        psi, inf, _ = gpu_run(g, psi0, 1e-4, 12, 6, V=V, order=order, boundary=boundary, tol=tol,
                              A_steps=A, precision=precision, step_mode=mode, shift=shift)
        outs[mode] = (psi, inf)
    a, ia = outs["passes"]
    op = oracle_op(g, V=V, order=order, boundary=ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC,
                   shift=shift)
    ref = psi0.copy()
    for s in range(6):
        op.A = tuple(A[s])
        ref, _ = lz.krylov_step(op, ref, 1e-4, 12, tol=tol)
    # (the mixed input carries 5 % random noise, which fills the whole spectrum)
    tol_ref = fp64_tol(6, 1e-4) if precision == "fp64" else \
        mixed_tol(6, 1e-4, max(hnorm(g, tuple(a), V, order) for a in A))
    for mode in modes[1:]:
        b, ib = outs[mode]
        assert ia.k_used == ib.k_used
        assert lz.rel_l2(b, a) <= (1e-13 if precision == "fp64" else 1e-6), mode
        assert lz.rel_l2(b, ref) <= tol_ref, mode


@pytest.mark.slow
def test_laser_packet_1024_full_size():
    """1024x1024, dx=0.05, m=20, dt=2e-4 in the sin^2 laser pulse, as the benchmark runs it:
    two steps element by element against the oracle, fifty against the closed form."""
    from paper_1407_7370_gb300.propagator import pulse_schedule
    cfg = wl.LASER_PACKET_1024
    g, p = cfg["grid"], cfg["pulse"]
    psi0 = wl.positive_energy_packet(g, p0=cfg["p0"], sigma_x=cfg["sigma_x"])
    dt, m, t0 = cfg["dt"], cfg["m"], 0.3
    A2 = pulse_schedule(t0, dt, 2, p.a0, p.omega, p.duration)
    out, info, _ = gpu_run(g, psi0, dt, m, 2, A_steps=A2)
    ref, oinf = lz.propagate(oracle_op(g), psi0.copy(), dt, m, 2, pulse=p, t0=t0)
    assert lz.rel_l2(out, ref) <= fp64_tol(2, dt)
    n = 50
    An = pulse_schedule(t0, dt, n, p.a0, p.omega, p.duration)
    out, info, _ = gpu_run(g, psi0, dt, m, n, A_steps=An)
    exact = free.propagate(oracle_op(g), psi0.copy(), dt, n, pulse=p, t0=t0)
    assert ham.norm(out - exact) <= info.cum_err + 1e-12 * ham.norm(exact)
    assert abs(ham.norm(out) - ham.norm(psi0)) <= 1e-12 * ham.norm(psi0)


_LONG_RUN = {}


def _long_run_exact(n, t0):
    """Closed-form propagation of the 1024^2 laser packet (cached: one CPU run
    serves both precisions)."""
    key = (n, t0)
    if key not in _LONG_RUN:
        cfg = wl.LASER_PACKET_1024
        g = cfg["grid"]
        psi0 = wl.positive_energy_packet(g, p0=cfg["p0"], sigma_x=cfg["sigma_x"])
        _LONG_RUN[key] = (psi0, free.propagate(oracle_op(g), psi0.copy(), cfg["dt"], n, pulse=cfg["pulse"],
                                               t0=t0))
    return _LONG_RUN[key]


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_laser_packet_1024_long_run_against_closed_form(precision):
    """200 steps (0.04 au of simulated time) of the benchmark's workload
    against the closed-form propagation in Fourier space, with the targets
    per unit of simulated time: 1e-10 (FP64) and 1e-5 (mixed)."""
    from paper_1407_7370_gb300.propagator import pulse_schedule
    cfg = wl.LASER_PACKET_1024
    g, p = cfg["grid"], cfg["pulse"]
    dt, m, t0, n = cfg["dt"], cfg["m"], 0.3, 200
    psi0, exact = _long_run_exact(n, t0)
    An = pulse_schedule(t0, dt, n, p.a0, p.omega, p.duration)
    shift = C * C if precision == "mixed" else 0.0
    out, info, _ = gpu_run(g, psi0, dt, m, n, A_steps=An, precision=precision, shift=shift)
    target = (1e-10 if precision == "fp64" else 1e-5) * n * dt
    assert lz.rel_l2(out, exact) <= target


# ---------------------------------------------------------------------------
# Mixed path: complex64 basis and FP32 stencil, FP64 scalars and state.
# Tolerance: relative L2 of psi at most 1e-5 per unit of simulated time
# against the FP64 oracle.  Runs too short for that to exceed one step's
# rounding get a floor:
#  * packets propagated with the shift s = m c^2 (packet_tol): the part of a
#    step that the mixed path holds in complex64 is the Krylov correction
#    psi' - C_1 psi; its rounding, 4 u32 times its size per step, measured on
#    the oracle's run (correction_sizes);
#  * states without the shift, or random spinors that fill the whole
#    spectrum (mixed_tol): their Krylov vectors carry every energy up to
#    ||H||, and the FP32 rounding of one application of exp(-iH dt) per step,
#    2 u32 ||H|| dt (u32 = 6e-8, ||H|| from the spectral bound of the
#    discrete operator), is the floor.
# ---------------------------------------------------------------------------
def hnorm(grid, A=(0.0, 0.0), V=None, order=2, c=137.036):
    pf = 1.0 if order == 2 else 1.3723
    px, py = pf / grid.dx + abs(A[0]), pf / grid.dy + abs(A[1])
    e = np.sqrt((c * c) ** 2 + c * c * (px * px + py * py))
    return e + (0.0 if V is None else float(np.max(np.abs(V))))


def mixed_tol(steps, dt, hn=None):
    floor = 0.0 if hn is None else 2 * 6e-8 * hn * dt * steps
    return max(1e-5 * steps * dt, floor)


def correction_size(psi, psi_next):
    """||psi' - <psi, psi'> psi / ||psi||^2|| / ||psi||: the part of one step
    that is not a multiple of psi (the Krylov correction)."""
    a = psi.reshape(-1)
    b = psi_next.reshape(-1)
    n2 = np.vdot(a, a).real
    return float(np.linalg.norm(b - (np.vdot(a, b) / n2) * a) / np.sqrt(n2))


def packet_tol(steps, dt, corrections):
    return max(1e-5 * steps * dt, 4 * 6e-8 * float(np.sum(corrections)))


def test_mixed_free_packet_64_full_run():
    cfg = wl.FREE_PACKET_64
    g = cfg["grid"]
    psi0 = wl.positive_energy_packet(g, p0=cfg["p0"], sigma_x=cfg["sigma_x"])
    out, info, _ = gpu_run(g, psi0, cfg["dt"], cfg["m"], cfg["steps"], precision="mixed")
    ref, _ = lz.propagate(oracle_op(g), psi0.copy(), cfg["dt"], cfg["m"], cfg["steps"])
    assert lz.rel_l2(out, ref) <= 1e-5 * cfg["steps"] * cfg["dt"]
    assert abs(ham.norm(out) - ham.norm(psi0)) <= 1e-9 * ham.norm(psi0)


@pytest.mark.parametrize("nx,ny,order,boundary,hasv,A", CASES[:4] + CASES[5:6])
def test_mixed_ragged_and_boundary_grids(nx, ny, order, boundary, hasv, A):
    g = wl.Grid(nx, ny, 0.1, 0.13)
    psi0 = wl.random_spinor(g, nx * 100 + ny) * 0.1
    V = wl.random_potential(g, 7, scale=20.0) if hasv else None
    dt, m, steps = 1e-4, 6, 3
    b = ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC
    out, info, _ = gpu_run(g, psi0, dt, m, steps, V=V, A=A, order=order, boundary=boundary,
                           precision="mixed")
    ref, _ = lz.propagate(oracle_op(g, V=V, A=A, order=order, boundary=b), psi0.copy(), dt, m, steps)
    assert lz.rel_l2(out, ref) <= mixed_tol(steps, dt, hnorm(g, A, V, order))


@pytest.mark.parametrize("mode", ["one_launch", "passes"])
def test_mixed_step_scalars_match_oracle(mode):
    g = wl.Grid(64, 48, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 5.0))
    V = wl.smoothed_coulomb(g, 3.0, 0.5)
    dt, m, s = 1e-4, 12, C * C
    out, info, _ = gpu_run(g, psi0, dt, m, 1, V=V, A=(4.0, -2.0), precision="mixed", shift=s,
                           step_mode=mode)
    ref, oi = lz.krylov_step(oracle_op(g, V=V, A=(4.0, -2.0), shift=s), psi0.copy(), dt, m)
    assert info.k_used == oi.k_used == m
    assert abs(info.energy - oi.energy) <= 1e-9 * abs(oi.energy)
    assert abs(info.norm - oi.norm) <= 1e-7 * oi.norm
    # alpha of H - s (the oracle's are of dt (H - s)), to 1e-6 of the largest |alpha|: the
    # packet's negative-energy admixture puts alpha_2 near -2 m c^2
    want = oi.alpha[:4] / dt
    diff = np.max(np.abs(np.asarray(info.alpha[:4]) - want))
    assert diff <= 1e-6 * np.max(np.abs(want)), (diff, info.alpha[:4], want)
    assert lz.rel_l2(out, ref) <= packet_tol(1, dt, [correction_size(psi0, ref)])


@pytest.mark.parametrize("p0", [(10.0, 0.0), (45.0, 10.0)])
def test_mixed_packet_long_run_at_target(p0):
    """A packet with the shift m c^2, 500 steps in a static field and a
    potential, against the oracle at the mixed target 1e-5 per unit time
    (no floor: the run is long enough for the target to exceed rounding)."""
    g = wl.Grid(96, 80, 0.05, 0.05)
    psi0 = wl.positive_energy_packet(g, p0=p0)
    V = wl.smoothed_coulomb(g, 2.0, 0.5)
    dt, m, steps, s = 2e-4, 16, 500, C * C
    out, info, _ = gpu_run(g, psi0, dt, m, steps, V=V, A=(2.0, -1.0), precision="mixed", shift=s)
    ref, _ = lz.propagate(oracle_op(g, V=V, A=(2.0, -1.0), shift=s), psi0.copy(), dt, m, steps)
    err = lz.rel_l2(out, ref)
    assert err <= 1e-5 * steps * dt, err


@pytest.mark.slow
def test_mixed_laser_packet_1024_against_closed_form():
    from paper_1407_7370_gb300.propagator import pulse_schedule
    cfg = wl.LASER_PACKET_1024
    g, p = cfg["grid"], cfg["pulse"]
    psi0 = wl.positive_energy_packet(g, p0=cfg["p0"], sigma_x=cfg["sigma_x"])
    dt, m, t0, n = cfg["dt"], cfg["m"], 0.3, 100
    An = pulse_schedule(t0, dt, n, p.a0, p.omega, p.duration)
    out, info, _ = gpu_run(g, psi0, dt, m, n, A_steps=An, precision="mixed")
    exact = free.propagate(oracle_op(g), psi0.copy(), dt, n, pulse=p, t0=t0)
    assert lz.rel_l2(out, exact) <= 1e-5 * n * dt
