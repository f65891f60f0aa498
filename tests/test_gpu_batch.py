"""Batched propagation: every problem of a batch against the CPU oracle.

The batch advances problems of different sizes together (one launch per
Lanczos iteration for all of them); each problem must match the oracle run
alone, within the same tolerances as the single-problem tests.
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import lanczos as lz
from paper_1407_7370_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def fp64_tol(steps, dt):
    return max(1e-10 * steps * dt, 1e-14 * steps)


def mixed_tol(steps, dt, hnorm):
    """States without the shift m c^2, or random spinors over the whole
    spectrum: 1e-5 per unit time, or FP32 rounding (storage and arithmetic)
    of one application of exp(-iH dt) per step, 2 u32 ||H|| dt, whichever is
    larger."""
    return max(1e-5 * steps * dt, 2 * 6e-8 * hnorm * dt * steps)


def correction_size(psi, psi_next):
    """Size of the Krylov correction of one step relative to ||psi||: the
    part of psi' that is not a multiple of psi, which the mixed path holds in
    complex64."""
    a = psi.reshape(-1)
    b = psi_next.reshape(-1)
    n2 = np.vdot(a, a).real
    return float(np.linalg.norm(b - (np.vdot(a, b) / n2) * a) / np.sqrt(n2))


def packet_tol(steps, dt, corrections):
    """Packets propagated with the shift m c^2: 1e-5 per unit time, or, for
    runs too short for that to exceed one step's rounding, 4 u32 times the
    size of each step's Krylov correction."""
    return max(1e-5 * steps * dt, 4 * 6e-8 * float(np.sum(corrections)))


def hnorm(grid, A, V=None, order=2, c=137.036):
    """Spectral radius bound of the discrete H (free part plus |V|)."""
    pf = 1.0 if order == 2 else 1.3723
    px, py = pf / grid.dx + np.max(np.abs(A[..., 0])), pf / grid.dy + np.max(np.abs(A[..., 1]))
    e = np.sqrt((c * c) ** 2 + c * c * (px * px + py * py))
    return e + (0.0 if V is None else np.max(np.abs(V)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_7370_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


GRIDS = [(64, 64, 0.1, 0.1), (37, 23, 0.1, 0.13), (16, 48, 0.12, 0.1), (96, 32, 0.1, 0.1),
         (7, 5, 0.2, 0.2), (128, 96, 0.08, 0.08)]


def _problem(k, g):
    grid = wl.Grid(*g)
    if k % 2 == 0:
        psi0 = wl.positive_energy_packet(grid, p0=(5.0 + 2 * k, 1.0))
    else:
        psi0 = 0.1 * wl.random_spinor(grid, 50 + k)
    V = wl.smoothed_coulomb(grid, 1.0 + k, 0.5) if k % 3 == 1 else None
    return grid, psi0, V


@pytest.mark.parametrize("precision,order,boundary,th,mode", [("fp64", 2, "periodic", 32, "auto"),
                                                               ("fp64", 4, "dirichlet", 32, "auto"),
                                                               ("fp64", 2, "periodic", 16, "auto"),
                                                               ("fp64", 4, "dirichlet", 16, "auto"),
                                                               ("mixed", 2, "periodic", 32, "auto"),
                                                               ("mixed", 2, "periodic", 16, "auto"),
                                                               ("mixed", 4, "dirichlet", 16, "auto"),
                                                               ("mixed", 2, "periodic", 16, "one_launch"),
                                                               ("mixed", 4, "dirichlet", 16, "one_launch"),
                                                               ("mixed", 2, "dirichlet", 16, "one_launch"),
                                                               ("mixed", 4, "periodic", 16, "one_launch")])
def test_batch_matches_oracle_per_problem(precision, order, boundary, th, mode):
    from paper_1407_7370_gb300 import BatchPropagator
    dt, m, steps = 1e-4, 8, 4
    bp = BatchPropagator(GRIDS, order=order, boundary=boundary, m_max=m, precision=precision)
    bp.set_launch_shape(th)
    bp.set_step_mode(mode)
    probs = [_problem(k, g) for k, g in enumerate(GRIDS)]
    rng = np.random.default_rng(7)
    A = rng.uniform(-20, 20, size=(steps, len(GRIDS), 2))
    for k, (grid, psi0, V) in enumerate(probs):
        bp.set_fields(k, None if V is None else torch.from_numpy(V).cuda())
    psis = [torch.from_numpy(p[1].copy()).cuda() for p in probs]
    infos = bp.steps(psis, steps, dt, m, A=A, info=True)
    b = ham.DIRICHLET if boundary == "dirichlet" else ham.PERIODIC
    for k, (grid, psi0, V) in enumerate(probs):
        op = ham.Operator(grid.nx, grid.ny, grid.dx, grid.dy, order=order, boundary=b, V=V)
        ref = psi0.copy()
        for s in range(steps):
            op.A = tuple(A[s, k])
            ref, oi = lz.krylov_step(op, ref, dt, m)
        err = lz.rel_l2(psis[k].cpu().numpy(), ref)
        tol = fp64_tol(steps, dt) if precision == "fp64" else \
            mixed_tol(steps, dt, hnorm(grid, A[:, k], V, order))
        assert err <= tol, (k, err)
        assert infos[k].k_used == oi.k_used


def test_batch_equals_single_problem_runs():
    from paper_1407_7370_gb300 import BatchPropagator, Propagator
    dt, m, steps = 1e-4, 10, 3
    bp = BatchPropagator(GRIDS, m_max=m)
    probs = [_problem(k, g) for k, g in enumerate(GRIDS)]
    for k, (grid, psi0, V) in enumerate(probs):
        bp.set_fields(k, None if V is None else torch.from_numpy(V).cuda(), A=(3.0, -1.0))
    psis = [torch.from_numpy(p[1].copy()).cuda() for p in probs]
    bp.steps(psis, steps, dt, m)
    for k, (grid, psi0, V) in enumerate(probs):
        single = Propagator(grid.nx, grid.ny, grid.dx, grid.dy, m_max=m)
        single.set_fields(None if V is None else torch.from_numpy(V).cuda(), A=(3.0, -1.0))
        p = torch.from_numpy(psi0.copy()).cuda()
        single.steps(p, steps, dt, m)
        assert lz.rel_l2(psis[k].cpu().numpy(), p.cpu().numpy()) <= fp64_tol(steps, dt)


def test_batch_kernel_launches_do_not_grow_with_problem_count():
    from paper_1407_7370_gb300 import BatchPropagator
    bp = BatchPropagator(GRIDS, m_max=6)
    probs = [_problem(k, g) for k, g in enumerate(GRIDS)]
    for k in range(len(GRIDS)):
        bp.set_fields(k)
    psis = [torch.from_numpy(p[1].copy()).cuda() for p in probs]
    bp.steps(psis, 2, 1e-4, 6, info=True)
    assert bp.kernel_launches == 1 + 2 * (6 + 2 + 1)
    # the mixed path runs every pass of every problem and the recombination
    # as one launch per step
    bm = BatchPropagator(GRIDS, m_max=6, precision="mixed")
    bm.set_step_mode("one_launch")
    for k in range(len(GRIDS)):
        bm.set_fields(k, shift=137.036 ** 2)
    psis = [torch.from_numpy(p[1].copy()).cuda() for p in probs]
    bm.steps(psis, 3, 1e-4, 6, info=True)
    assert bm.kernel_launches == 1 + 3 * 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_direct_launches(precision):
    from paper_1407_7370_gb300 import BatchPropagator
    probs = [_problem(k, g) for k, g in enumerate(GRIDS)]
    A = np.random.default_rng(3).uniform(-5, 5, size=(6, len(GRIDS), 2))
    outs = []
    for graphs in (True, False):
        bp = BatchPropagator(GRIDS, m_max=8, precision=precision)
        bp.use_graphs(graphs)
        for k, (grid, psi0, V) in enumerate(probs):
            bp.set_fields(k, None if V is None else torch.from_numpy(V).cuda())
        psis = [torch.from_numpy(p[1].copy()).cuda() for p in probs]
        bp.steps(psis, 6, 1e-4, 8, A=A)
        outs.append([p.cpu().numpy() for p in psis])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_autotune_leaves_states_and_picks_a_shape(tmp_path, monkeypatch):
    from paper_1407_7370_gb300 import BatchPropagator
    monkeypatch.setenv("DIRAC_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    probs = [_problem(k, g) for k, g in enumerate(GRIDS)]
    bp = BatchPropagator(GRIDS, m_max=8, precision="mixed")
    for k, (grid, psi0, V) in enumerate(probs):
        bp.set_fields(k, None if V is None else torch.from_numpy(V).cuda())
    psis = [torch.from_numpy(p[1].copy()).cuda() for p in probs]
    r = bp.autotune(psis, 1e-4, 8, steps=2)
    assert r["tile_height"] in (16, 32) and r["candidates"] >= 2 and not r["from_cache"]
    for p, (grid, psi0, V) in zip(psis, probs):
        assert np.array_equal(p.cpu().numpy(), psi0)
    # the choice is reused from the cache file by an identical batch
    bp2 = BatchPropagator(GRIDS, m_max=8, precision="mixed")
    r2 = bp2.autotune(psis, 1e-4, 8, steps=2)
    assert r2["from_cache"] and r2["tile_height"] == r["tile_height"]
    # and stepping after tuning still matches the oracle
    for k in range(len(GRIDS)):
        bp.set_fields(k, None if probs[k][2] is None else torch.from_numpy(probs[k][2]).cuda())
    bp.steps(psis, 2, 1e-4, 8)
    grid, psi0, V = probs[0]
    op = ham.Operator(grid.nx, grid.ny, grid.dx, grid.dy, V=V)
    ref, _ = lz.propagate(op, psi0.copy(), 1e-4, 8, 2)
    assert lz.rel_l2(psis[0].cpu().numpy(), ref) <= mixed_tol(2, 1e-4, hnorm(grid, np.zeros((1, 2)), V))


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_256_full_size_sampled(precision):
    """The batched workload at its full size (256 packets on 128^2..512^2
    grids, m = 16, laser amplitudes up to 100 au), autotuned and replayed as
    a graph as the benchmark runs it: one problem of every grid size against
    the oracle run alone (its own step means of the pulse), over 20 steps
    (the oracle runs in spawned processes while the GPU works)."""
    import concurrent.futures
    import multiprocessing

    from paper_1407_7370_gb300 import BatchPropagator
    from paper_1407_7370_gb300.propagator import pulse_sin2_mean
    cfg = wl.BATCH_256
    grids, p0s, a0s = wl.batch_packets(cfg["n"])
    m, dt, n, pulse = cfg["m"], cfg["dt"], cfg["n"], cfg["pulse"]
    steps, C2 = 20, 137.036 ** 2
    t0 = 0.5   # mid-pulse, where A_x reaches a few au
    sample = [next(k for k, g in enumerate(grids) if g.nx == side) for side in (128, 256, 384, 512)]
    psi0 = [wl.positive_energy_packet(g, p0=(float(p), 0.0)) for g, p in zip(grids, p0s)]
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=len(sample), mp_context=ctx) as pool:
        futs = {}
        for k in sample:
            g = grids[k]
            op = ham.Operator(g.nx, g.ny, g.dx, g.dy, shift=C2)
            pk = wl.SinSquaredPulse(float(a0s[k]), pulse.omega, pulse.duration)
            futs[k] = pool.submit(lz.propagate, op, psi0[k].copy(), dt, m, steps, pk, t0)
        base = np.array([pulse_sin2_mean(t0 + k * dt, dt, 1.0, pulse.omega, pulse.duration)
                         for k in range(steps + 1)])
        A = np.zeros((steps + 1, n, 2))
        A[:, :, 0] = base[:, None] * a0s[None, :]
        bp = BatchPropagator([(g.nx, g.ny, g.dx, g.dy) for g in grids], m_max=m, precision=precision)
        for k in range(n):
            bp.set_fields(k, shift=C2)
        psis = [torch.from_numpy(p.copy()).cuda() for p in psi0]
        bp.autotune(psis, dt, m, A=A[:3], steps=3)
        bp.steps(psis, steps, dt, m, A=A[:steps])
        for k in sample:
            ref, _ = futs[k].result()
            err = lz.rel_l2(psis[k].cpu().numpy(), ref)
            tol = fp64_tol(steps, dt) if precision == "fp64" else 1e-5 * steps * dt
            assert err <= tol, (k, grids[k].nx, err, tol)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_per_problem_stopping(precision):
    """Problems of one batch stop at their own Krylov dimension: an exact
    plane-wave eigenvector breaks down after one iteration (FP64), the zero
    state is a trivial step, and with tol > 0 a slow and a fast packet stop
    at different k (Eq. 18) -- each as the oracle run alone does."""
    from paper_1407_7370_gb300 import BatchPropagator
    from tests.test_oracle_hamiltonian import plane_wave_eigpair
    grids = [wl.Grid(32, 24, 0.1, 0.1), wl.Grid(48, 40, 0.1, 0.1), wl.Grid(40, 40, 0.05, 0.05),
             wl.Grid(17, 9, 0.1, 0.1)]
    pw, _ = plane_wave_eigpair(32, 24, 0.1, 0.1, 2, 1, 2, (0.0, 0.0), 0.0)
    states = [pw, wl.positive_energy_packet(grids[1], p0=(0.5, 0.0), sigma_x=2.0),
              wl.positive_energy_packet(grids[2], p0=(40.0, 10.0), sigma_x=0.3),
              np.zeros((9, 17, 2), complex)]
    dt, m, tol, steps = 2e-4, 16, 1e-9, 2
    shift = 137.036 ** 2 if precision == "mixed" else 0.0
    bp = BatchPropagator([(g.nx, g.ny, g.dx, g.dy) for g in grids], m_max=m, precision=precision)
    for k in range(len(grids)):
        bp.set_fields(k, shift=shift)
    psis = [torch.from_numpy(s.copy()).cuda() for s in states]
    infos = bp.steps(psis, steps, dt, m, tol=tol, info=True)
    assert not np.any(psis[3].cpu().numpy()) and infos[3].k_used == 1
    if precision == "fp64":   # FP32 stencil rounding leaves beta_1 ~ u32 ||H||: no exact breakdown
        assert infos[0].k_used == 1 and infos[0].breakdown
    ks = []
    corrs = {}
    for k in range(3):
        g = grids[k]
        op = ham.Operator(g.nx, g.ny, g.dx, g.dy, shift=shift)
        ref = states[k].copy()
        corrs[k] = []
        for _ in range(steps):
            nxt, oi = lz.krylov_step(op, ref, dt, m, tol=tol)
            corrs[k].append(correction_size(ref, nxt))
            ref = nxt
        out = psis[k].cpu().numpy()
        if precision == "fp64":
            assert infos[k].k_used == oi.k_used, (k, infos[k].k_used, oi.k_used)
            assert lz.rel_l2(out, ref) <= fp64_tol(steps, dt)
        else:
            if k > 0:
                assert abs(infos[k].k_used - oi.k_used) <= 1
            if k == 0:   # an exact eigenvector of the FP64 operator: beta_1 is FP32 rounding
                assert lz.rel_l2(out, ref) <= mixed_tol(steps, dt, hnorm(g, np.zeros((1, 2))))
            else:        # packets with the shift m c^2
                assert lz.rel_l2(out, ref) <= packet_tol(steps, dt, corrs[k])
        ks.append(infos[k].k_used)
    assert ks[1] < ks[2]      # the fast, narrow packet needs a larger Krylov space


@pytest.mark.slow
def test_batch_sampled_problems_500_steps_at_target():
    """Eight problems of the batched workload -- the fastest packet (largest
    p0), the strongest field (largest A0) and six spread over the p0 range --
    advanced together on the mixed path for 500 steps (0.1 au, mid-pulse)
    against the oracle at the mixed target, 1e-5 relative L2 per unit time,
    with no floor.  They run on the workload's smallest grid side (128^2,
    dx = 0.05), which the oracle finishes in about half a minute per problem
    (run in parallel, in freshly spawned processes)."""
    import concurrent.futures
    import multiprocessing
    import os

    from paper_1407_7370_gb300 import BatchPropagator
    from paper_1407_7370_gb300.propagator import pulse_sin2_mean
    cfg = wl.BATCH_256
    _, p0s, a0s = wl.batch_packets(cfg["n"])
    order = np.argsort(p0s)
    pick = [int(np.argmax(p0s)), int(np.argmax(a0s))]
    for q in (0.05, 0.25, 0.45, 0.65, 0.8, 0.95):
        k = int(order[int(q * (len(order) - 1))])
        if k not in pick:
            pick.append(k)
    pick = pick[:8]
    m, dt, steps, t0, C2 = cfg["m"], cfg["dt"], 500, 0.5, 137.036 ** 2
    g = wl.Grid(128, 128, 0.05, 0.05)
    pulse = cfg["pulse"]
    psi0 = [wl.positive_energy_packet(g, p0=(float(p0s[k]), 0.0)) for k in pick]
    # the oracle runs first, in spawned processes, while the GPU works
    ctx = multiprocessing.get_context("spawn")
    workers = min(len(pick), max(1, (os.cpu_count() or 2) - 1))
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool:
        futs = []
        for j, k in enumerate(pick):
            op = ham.Operator(g.nx, g.ny, g.dx, g.dy, shift=C2)
            pk = wl.SinSquaredPulse(float(a0s[k]), pulse.omega, pulse.duration)
            futs.append(pool.submit(lz.propagate, op, psi0[j].copy(), dt, m, steps, pk, t0))
        base = np.array([pulse_sin2_mean(t0 + s * dt, dt, 1.0, pulse.omega, pulse.duration)
                         for s in range(steps)])
        A = np.zeros((steps, len(pick), 2))
        A[:, :, 0] = base[:, None] * a0s[pick][None, :]
        outs = {}
        for mode in ("passes", "one_launch"):   # both launch forms of the mixed path
            bp = BatchPropagator([(g.nx, g.ny, g.dx, g.dy)] * len(pick), m_max=m, precision="mixed")
            bp.set_step_mode(mode)
            for j in range(len(pick)):
                bp.set_fields(j, shift=C2)
            psis = [torch.from_numpy(p.copy()).cuda() for p in psi0]
            bp.steps(psis, steps, dt, m, A=A, info=True)
            outs[mode] = [p.cpu().numpy() for p in psis]
            bp.close()
        refs = [f.result()[0] for f in futs]
    target = 1e-5 * steps * dt
    for mode, out in outs.items():
        errs = [lz.rel_l2(a, r) for a, r in zip(out, refs)]
        print("mixed (%s) vs oracle after %d steps (p0, A0, rel L2):" % (mode, steps),
              [(round(float(p0s[k]), 1), round(float(a0s[k]), 1), "%.2e" % e) for k, e in zip(pick, errs)])
        assert max(errs) <= target, (mode, errs, target)
