"""Parity of the adjoint (dirac_adjoint_gradient) with the CPU oracle's
forward-mode Frechet gradients, with central finite differences of the GPU
forward map, and with invariances; the autograd front end.

Tolerances: the oracle uses the exact exponential; the GPU the Krylov one with
m = 16 at |dt| ||H - s|| < 1, whose error (Eq. 18) is below 1e-18, and sums in
another order, so gradients agree to ~1e-10 relative to their largest entry.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import hamiltonian as ham
from paper_1407_7370_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C = 137.036


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_7370_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def small_case(nx=6, ny=5, dx=0.4, z=2.0, seed=3, nsteps=4):
    g = wl.Grid(nx, ny, dx, dx)
    V = wl.soft_core(g, z) + 0.3 * wl.random_potential(g, seed, scale=1.0)
    op = ham.Operator(nx, ny, dx, dx, V=V, shift=C * C)
    psi0 = wl.positive_energy_packet(g, p0=(2.0, 1.0), sigma_x=0.8)
    phi = wl.normalise(wl.random_spinor(g, seed + 1), g)
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, (nsteps, 2))
    return g, op, psi0, phi, A


def lib_W(nsteps, dt, ncoef, duration):
    """The library's closed-form step means of the sine basis (the GPU side's input)."""
    from paper_1407_7370_gb300.propagator import pulse_sine_basis_means
    return pulse_sine_basis_means(nsteps, dt, ncoef, duration)


def gpu_prop(g, V, m=16, order=2, boundary="periodic"):
    from paper_1407_7370_gb300 import Propagator
    p = Propagator(g.nx, g.ny, g.dx, g.dy, order=order, boundary=boundary, m_max=m)
    p.set_fields(dev(V), shift=C * C)
    return p


@pytest.mark.parametrize("kind", ["px", "proj"])
def test_adjoint_matches_oracle_per_site_and_step(kind):
    g, op, psi0, phi, A = small_case()
    dt = 2e-5
    p = gpu_prop(g, op.V)
    res = p.adjoint_gradient(dev(psi0), A.shape[0], dt, 16, A, observable=kind, phi=dev(phi),
                             checkpoint_every=3)
    ref = adj.gradient(op, psi0, dt, A, kind, phi)
    assert abs(res.loss - ref.loss) <= 1e-12 * abs(ref.loss)
    dV = res.dV.cpu().numpy().reshape(-1)
    assert np.max(np.abs(dV - ref.dV)) <= 1e-9 * np.max(np.abs(ref.dV))
    assert np.max(np.abs(res.dA - ref.dA)) <= 1e-9 * np.max(np.abs(ref.dA))


@pytest.mark.parametrize("kind,order,boundary", [("px", 2, "periodic"), ("proj", 4, "dirichlet"),
                                                 ("px", 4, "dirichlet")])
def test_adjoint_contracted_with_random_direction_matches_oracle_jvp(kind, order, boundary):
    """A 40x20 grid (several warps and blocks per row, ragged in both
    directions), where the oracle runs one forward-mode sweep along a random
    direction instead of one per site: the GPU's reverse-mode gradient
    contracted with that direction must give the same derivative."""
    g, op, psi0, phi, A = small_case(40, 20, 0.3, nsteps=3)
    op = ham.Operator(g.nx, g.ny, g.dx, g.dy, order=order,
                      boundary=ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC,
                      V=op.V, shift=C * C)
    dt = 2e-5
    rng = np.random.default_rng(5)
    dV = rng.standard_normal((g.ny, g.nx))
    dA = rng.standard_normal(A.shape)
    p = gpu_prop(g, op.V, order=order, boundary=boundary)
    res = p.adjoint_gradient(dev(psi0), A.shape[0], dt, 16, A, observable=kind, phi=dev(phi),
                             checkpoint_every=2)
    L, d_ref = adj.jvp(op, psi0, dt, A, kind, phi, dV=dV, dA=dA)
    d_gpu = float(np.sum(res.dV.cpu().numpy() * dV) + np.sum(res.dA * dA))
    scale = float(np.sum(np.abs(res.dV.cpu().numpy() * dV)) + np.sum(np.abs(res.dA * dA)))
    assert abs(res.loss - L) <= 1e-12 * abs(L)
    assert abs(d_gpu - d_ref) <= 1e-10 * scale, (d_gpu, d_ref, scale)


def test_adjoint_blocks_and_pulse_coefficients_match_oracle():
    g, op, psi0, phi, A = small_case(8, 6, 0.35, nsteps=5)
    dt = 2e-5
    coef = np.array([0.7, -0.4, 0.2])
    W = adj.sine_basis_means(5, dt, 3, 5 * dt)
    Wg = lib_W(5, dt, 3, 5 * dt)
    Ag = A.copy()
    A[:, 0] = W @ coef
    Ag[:, 0] = Wg @ coef
    p = gpu_prop(g, op.V)
    res = p.adjoint_gradient(dev(psi0), 5, dt, 16, Ag, observable="proj", phi=dev(phi),
                             checkpoint_every=2, block=(2, 2), W=Wg)
    ref = adj.gradient(op, psi0, dt, A, "proj", phi)
    pooled = ref.dV.reshape(6, 8).reshape(3, 2, 4, 2).sum(axis=(1, 3))
    assert np.max(np.abs(res.dV.cpu().numpy() - pooled)) <= 1e-9 * np.max(np.abs(pooled))
    da_ref = W.T @ ref.dA[:, 0]
    assert np.max(np.abs(res.da - da_ref)) <= 1e-9 * np.max(np.abs(da_ref))


def test_checkpoint_interval_does_not_change_the_result():
    """Only the rounding may differ: a multi-step forward call takes one
    Chebyshev interval for all its steps (from their largest |A|), a
    one-step call its own."""
    g, op, psi0, phi, A = small_case(nsteps=7)
    p = gpu_prop(g, op.V)
    runs = [p.adjoint_gradient(dev(psi0), 7, 2e-5, 16, A, observable="px", checkpoint_every=k)
            for k in (1, 3, 7)]
    base_dV = runs[0].dV.cpu().numpy()
    for r in runs[1:]:
        assert abs(r.loss - runs[0].loss) <= 1e-13 * abs(runs[0].loss)
        assert np.max(np.abs(r.dV.cpu().numpy() - base_dV)) <= 1e-11 * np.max(np.abs(base_dV))
        # the A gradients are sums over sites with much cancellation
        assert np.max(np.abs(r.dA - runs[0].dA)) <= 1e-9 * np.max(np.abs(runs[0].dA))
    # the same call twice is bitwise the same
    again = p.adjoint_gradient(dev(psi0), 7, 2e-5, 16, A, observable="px", checkpoint_every=3)
    assert again.loss == runs[1].loss and torch.equal(again.dV, runs[1].dV)
    assert np.array_equal(again.dA, runs[1].dA)


@pytest.mark.parametrize("kind", ["px", "proj"])
def test_adjoint_matches_gpu_finite_differences(kind):
    g = wl.Grid(48, 40, 0.1, 0.1)
    V = wl.smoothed_coulomb(g, 2.0, 0.5)
    psi0 = wl.positive_energy_packet(g, p0=(3.0, 0.0), sigma_x=0.6)
    phi = wl.normalise(wl.positive_energy_packet(g, p0=(0.0, 0.0), sigma_x=0.5), g)
    nsteps, dt = 12, 2e-4
    W = lib_W(nsteps, dt, 4, nsteps * dt)
    coef = np.array([30.0, -10.0, 5.0, 2.0])
    A = np.zeros((nsteps, 2))
    A[:, 0] = W @ coef
    p = gpu_prop(g, V, m=20)
    res = p.adjoint_gradient(dev(psi0), nsteps, dt, 20, A, observable=kind, phi=dev(phi),
                             checkpoint_every=5, block=(8, 8), W=W)

    def loss(Vx, Ax):
        q = gpu_prop(g, Vx, m=20)
        return q.adjoint_gradient(dev(psi0), nsteps, dt, 20, Ax, observable=kind, phi=dev(phi),
                                  grad_V=False, grad_A=False).loss

    h = 1e-4
    dV = res.dV.cpu().numpy()

    def close(fd, gr):   # FD truncation ~h^2, rounding of L ~1e-13 |L| / h
        return abs(fd - gr) <= 1e-5 * abs(gr) + 1e-13 * abs(res.loss) / h
    for (by, bx) in ((2, 3), (0, 0)):
        Vp, Vm = V.copy(), V.copy()
        Vp[8 * by:8 * by + 8, 8 * bx:8 * bx + 8] += h
        Vm[8 * by:8 * by + 8, 8 * bx:8 * bx + 8] -= h
        fd = (loss(Vp, A) - loss(Vm, A)) / (2 * h)
        assert close(fd, dV[by, bx]), (by, bx, fd, dV[by, bx])
    for k in (0, 2):
        e = np.zeros(4)
        e[k] = h
        Ap, Am = A.copy(), A.copy()
        Ap[:, 0] = W @ (coef + e)
        Am[:, 0] = W @ (coef - e)
        fd = (loss(V, Ap) - loss(V, Am)) / (2 * h)
        assert close(fd, res.da[k]), (k, fd, res.da[k])


def test_uniform_potential_gradient_vanishes_on_gpu():
    g, op, psi0, phi, A = small_case(10, 8, 0.3, nsteps=6)
    p = gpu_prop(g, op.V)
    res = p.adjoint_gradient(dev(psi0), 6, 2e-4, 16, A, observable="proj", phi=dev(phi))
    dV = res.dV.cpu().numpy()
    assert abs(dV.sum()) <= 1e-10 * np.abs(dV).sum()


def test_autograd_front_end():
    from paper_1407_7370_gb300.autograd import AdjointSetup, propagated_observable
    g = wl.Grid(16, 12, 0.2, 0.2)
    psi0 = dev(wl.positive_energy_packet(g, p0=(2.0, 0.0), sigma_x=0.5))
    nsteps, dt = 6, 1e-4
    W = lib_W(nsteps, dt, 2, nsteps * dt)
    setup = AdjointSetup(g.nx, g.ny, g.dx, g.dy, psi0, dt, 16, nsteps, W, observable="px",
                         block=(4, 4), checkpoint_every=2, shift=C * C)
    Vb = torch.tensor(np.random.default_rng(0).uniform(-2, 0, (3, 4)), dtype=torch.float64,
                      device="cuda", requires_grad=True)
    coef = torch.tensor([20.0, -5.0], dtype=torch.float64, device="cuda", requires_grad=True)
    L = propagated_observable(Vb, coef, setup)
    gV, ga = torch.autograd.grad(2.0 * L, (Vb, coef))
    # the same numbers straight from the library
    V = Vb.detach().repeat_interleave(4, 0).repeat_interleave(4, 1).contiguous()
    prop = gpu_prop(g, V.cpu().numpy())
    A = np.zeros((nsteps, 2))
    A[:, 0] = W @ coef.detach().cpu().numpy()
    res = prop.adjoint_gradient(psi0, nsteps, dt, 16, A, observable="px", checkpoint_every=2,
                                block=(4, 4), W=W)
    assert abs(L.item() - res.loss) == 0.0
    assert torch.allclose(gV, 2.0 * res.dV, rtol=0, atol=0)
    assert np.allclose(ga.cpu().numpy(), 2.0 * res.da, rtol=0, atol=0)


def bound_state_guess(g):
    """A normalised positive-energy Gaussian of width 0.7 au at rest: close to
    the ground state of the smoothed Coulomb well (the projector is fixed, so
    any state serves the gradient check)."""
    return dev(wl.positive_energy_packet(g, p0=(0.0, 0.0), sigma_x=0.7))


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["px", "proj"])
def test_adjoint_full_size_1024_against_finite_differences(kind):
    """1024x1024, dx = 0.05, m = 16, 2000 steps of 2e-4, checkpoints every 50
    steps; V constant on 4x4 blocks (a 256x256 grid, the smoothed Coulomb
    potential Z = 1, a = 0.5), A_x a 64-term sine series over the run; start
    in the projector's state.  Central differences (h = 1e-6) at sampled
    parameters."""
    g = wl.Grid(1024, 1024, 0.05, 0.05)
    V = wl.smoothed_coulomb(g, 1.0, 0.5)
    phi = bound_state_guess(g)
    Vb = V.reshape(256, 4, 256, 4).mean(axis=(1, 3))
    Vs = np.repeat(np.repeat(Vb, 4, 0), 4, 1)
    nsteps, dt = 2000, 2e-4
    W = lib_W(nsteps, dt, 64, nsteps * dt)
    coef = np.random.default_rng(5).uniform(-1.0, 1.0, 64) * 5.0 / (1.0 + np.arange(64))
    A = np.zeros((nsteps, 2))
    A[:, 0] = W @ coef
    p = gpu_prop(g, Vs, m=16)
    res = p.adjoint_gradient(phi, nsteps, dt, 16, A, observable=kind, phi=phi, checkpoint_every=50,
                             block=(4, 4), W=W)
    assert res.dV.shape == (256, 256)
    dV = res.dV.cpu().numpy()

    def loss(Vx, Ax):
        q = gpu_prop(g, Vx, m=16)
        out = q.adjoint_gradient(phi, nsteps, dt, 16, Ax, observable=kind, phi=phi,
                                 grad_V=False, grad_A=False).loss
        q.close()
        return out

    h = 1e-6

    def close(fd, gr):   # rounding of L over 2000 steps ~1e-13 |L|, divided by h
        return abs(fd - gr) <= 1e-4 * abs(gr) + 2e-13 * max(abs(res.loss), 1.0) / h

    iy, ix = np.unravel_index(np.argmax(np.abs(dV)), dV.shape)
    Vp, Vm = Vs.copy(), Vs.copy()
    Vp[4 * iy:4 * iy + 4, 4 * ix:4 * ix + 4] += h
    Vm[4 * iy:4 * iy + 4, 4 * ix:4 * ix + 4] -= h
    fd = (loss(Vp, A) - loss(Vm, A)) / (2 * h)
    assert close(fd, dV[iy, ix]), (iy, ix, fd, dV[iy, ix])
    for k in (0, 5):
        e = np.zeros(64)
        e[k] = h
        Ap, Am = A.copy(), A.copy()
        Ap[:, 0] = W @ (coef + e)
        Am[:, 0] = W @ (coef - e)
        fd = (loss(Vs, Ap) - loss(Vs, Am)) / (2 * h)
        assert close(fd, res.da[k]), (k, fd, res.da[k])
