"""The allocation-free step, dirac_lanczos_step_noalloc, against the regular step.

Some callers cannot let a library allocate device memory -- a host framework
that owns every device allocation, a memory budget fixed before the run, a
per-step loop where an allocation's latency or failure is not acceptable.
For them the library offers one step that keeps its whole workspace in a
static device array.  These tests call it through the C ABI twice in a row
and compare each result with the regular context-based step launched one
pass at a time, within the FP64 parity tolerance used by the other GPU
tests, over the operator's variants (potential or none, stencil order 2 and
4, periodic and Dirichlet boundaries, A_y zero or not, a fixed Krylov
dimension and an adaptive one, forward and backward steps); and they check
that repeated calls leave the device's free memory unchanged.  The file name
sorts last so that a run stopping at the first failure has run everything
else first.
"""
import ctypes

import numpy as np
import pytest

from paper_1407_7370_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def fp64_tol(steps, dt):
    return max(1e-10 * steps * abs(dt), 1e-14 * steps)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def lib():
    from paper_1407_7370_gb300 import build
    from paper_1407_7370_gb300 import _native as nat
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return nat


# (with V, stencil order, boundary, A, tol, dt)
CASES = [
    (True, 2, "periodic", (4.0, -2.0), 0.0, 1e-4),
    (False, 2, "periodic", (4.0, 0.0), 0.0, 1e-4),
    (True, 4, "periodic", (0.0, 3.0), 0.0, 1e-4),
    (True, 2, "dirichlet", (2.0, 1.0), 0.0, 1e-4),
    (False, 4, "dirichlet", (0.0, 0.0), 0.0, 1e-4),
    (True, 2, "periodic", (4.0, -2.0), 1e-8, 1e-4),
    (False, 2, "periodic", (1.0, 0.0), 1e-8, -1e-4),
    (True, 4, "dirichlet", (3.0, -1.0), 0.0, -1e-4),
]


@pytest.mark.parametrize("with_v,order,boundary,A,tol,dt", CASES)
def test_noalloc_step_matches_regular_step_on_two_calls(lib, with_v, order, boundary, A, tol, dt):
    from paper_1407_7370_gb300 import Propagator
    g = wl.Grid(64, 48, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(10.0, 5.0))
    V = torch.from_numpy(wl.smoothed_coulomb(g, 3.0, 0.5)).cuda() if with_v else None
    m = 12

    prop = Propagator(g.nx, g.ny, g.dx, g.dy, m_max=m, order=order, boundary=boundary)
    prop.set_step_mode("passes")
    prop.set_fields(V, A=A)
    psi_r = torch.from_numpy(psi0.copy()).cuda()

    bnd = lib.PERIODIC if boundary == "periodic" else lib.DIRICHLET
    prob = lib.ProblemC(g.nx, g.ny, g.dx, g.dy, 1.0, 137.036, order, bnd,
                        ctypes.c_void_p(V.data_ptr()) if with_v else None, A[0], A[1], 0.0)
    psi_n = torch.from_numpy(psi0.copy()).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = lib.lib()
    for call in (1, 2):
        ref = prop.step(psi_r, dt, m, tol=tol, info=True)
        info = lib.StepInfoC()
        lib.check(L.dirac_lanczos_step_noalloc(ctypes.byref(prob), ctypes.c_void_p(psi_n.data_ptr()),
                                               dt, m, tol, stream, ctypes.byref(info)))
        a, b = psi_n.cpu().numpy(), psi_r.cpu().numpy()
        assert rel_l2(a, b) <= fp64_tol(call, dt), (call, rel_l2(a, b))
        assert info.k_used == ref.k_used
        if tol == 0.0:
            assert info.k_used == m
        else:
            assert info.k_used < m
        assert abs(info.energy - ref.energy) <= 1e-12 * abs(ref.energy)
        assert abs(info.err_est - ref.err_est) <= 1e-6 * ref.err_est + 1e-14 * ref.norm
    prop.close()


def test_noalloc_forward_then_backward_returns(lib):
    g = wl.Grid(40, 36, 0.1, 0.1)
    psi0 = wl.positive_energy_packet(g, p0=(8.0, -3.0))
    prob = lib.ProblemC(g.nx, g.ny, g.dx, g.dy, 1.0, 137.036, 2, lib.PERIODIC, None, 2.0, 1.0, 0.0)
    psi = torch.from_numpy(psi0.copy()).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = lib.lib()
    for dt in (1e-4, -1e-4):
        lib.check(L.dirac_lanczos_step_noalloc(ctypes.byref(prob), ctypes.c_void_p(psi.data_ptr()),
                                               dt, 16, 0.0, stream, None))
    torch.cuda.synchronize()
    assert rel_l2(psi.cpu().numpy(), psi0) <= 1e-12


def test_noalloc_calls_leave_free_memory_unchanged(lib):
    g = wl.Grid(48, 40, 0.1, 0.1)
    psi = torch.from_numpy(wl.positive_energy_packet(g, p0=(5.0, 0.0))).cuda()
    V = torch.from_numpy(wl.smoothed_coulomb(g, 2.0, 0.5)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = lib.lib()
    info = lib.StepInfoC()
    for with_v in (False, True):
        prob = lib.ProblemC(g.nx, g.ny, g.dx, g.dy, 1.0, 137.036, 2, lib.PERIODIC,
                            ctypes.c_void_p(V.data_ptr()) if with_v else None, 1.0, 0.0, 0.0)
        # the first call may load the module's data on this device
        lib.check(L.dirac_lanczos_step_noalloc(ctypes.byref(prob), ctypes.c_void_p(psi.data_ptr()),
                                               1e-4, 10, 0.0, stream, ctypes.byref(info)))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(5):
            lib.check(L.dirac_lanczos_step_noalloc(ctypes.byref(prob), ctypes.c_void_p(psi.data_ptr()),
                                                   1e-4, 10, 0.0, stream, None))
        lib.check(L.dirac_lanczos_step_noalloc(ctypes.byref(prob), ctypes.c_void_p(psi.data_ptr()),
                                               1e-4, 10, 0.0, stream, ctypes.byref(info)))
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (with_v, free0, free1)


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    L = lib.lib()
    assert L.dirac_noalloc_scratch_bytes() == 8 << 20
    psi = torch.zeros((512, 512, 2), dtype=torch.complex128, device="cuda")
    prob = lib.ProblemC(512, 512, 0.05, 0.05, 1.0, 137.036, 2, lib.PERIODIC, None, 0.0, 0.0, 0.0)
    st = L.dirac_lanczos_step_noalloc(ctypes.byref(prob), ctypes.c_void_p(psi.data_ptr()), 1e-4, 10,
                                      0.0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                      None)
    assert st == lib.EINVAL
    assert b"scratch" in L.dirac_last_error()
