"""CPU-side checks of the C ABI: the library builds, loads, exports every
function that include/dirac.h declares, and its host-only pieces behave."""
import ctypes
import os

import pytest

from paper_1407_7370_gb300 import _native as nat
from paper_1407_7370_gb300 import build as bld
from paper_1407_7370_gb300 import workloads as wl


@pytest.fixture(scope="session")
def lib():
    bld.build()
    return nat.lib()


def test_every_declared_function_is_exported(lib):
    names = nat.header_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in range(6):
        assert lib.dirac_status_string(s)
    assert lib.dirac_status_string(0) == b"ok"


def test_pulse_mean_matches_oracle_quadrature(lib):
    from oracle import fields
    p = wl.SinSquaredPulse(50.0, 0.05, 1.0)
    for t0 in (-3e-4, -1e-4, 0.0, 0.25, 0.77, 0.9999, 1.0, 1.5):
        a = lib.dirac_pulse_sin2_mean(t0, 2e-4, p.a0, p.omega, p.duration)
        b = fields.step_mean(p, t0, 2e-4)
        assert abs(a - b) <= 1e-13 * p.a0


def test_sine_basis_means_match_oracle(lib):
    import numpy as np
    from oracle import adjoint as adj
    from paper_1407_7370_gb300.propagator import pulse_sine_basis_means
    for nsteps, dt, k, T in ((7, 0.01, 5, 0.37), (2000, 2e-4, 64, 0.4)):
        W = pulse_sine_basis_means(nsteps, dt, k, T)
        assert np.max(np.abs(W - adj.sine_basis_means(nsteps, dt, k, T))) <= 1e-12


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    ctx = ctypes.c_void_p()
    bad = [
        (0, 8, 0.1, 0.1, 1.0, 137.0, 2, 0, 0, 10),
        (8, 8, -0.1, 0.1, 1.0, 137.0, 2, 0, 0, 10),
        (8, 8, 0.1, 0.1, 1.0, 0.0, 2, 0, 0, 10),
        (8, 8, 0.1, 0.1, 1.0, 137.0, 3, 0, 0, 10),
        (8, 8, 0.1, 0.1, 1.0, 137.0, 2, 5, 0, 10),
        (8, 8, 0.1, 0.1, 1.0, 137.0, 2, 0, 7, 10),
        (8, 8, 0.1, 0.1, 1.0, 137.0, 2, 0, 0, 0),
        (8, 8, 0.1, 0.1, 1.0, 137.0, 2, 0, 0, 33),
    ]
    for args in bad:
        assert lib.dirac_create(ctypes.byref(ctx), *args, None) == nat.EINVAL
        assert lib.dirac_last_error()
        assert not ctx.value


def test_binding_constants_match_the_header():
    import re
    text = open(nat.HEADER).read()
    defs = dict(re.findall(r"#define\s+(DIRAC_\w+)\s+(-?\d+)", text))
    for name, value in (("DIRAC_KERNEL_KINDS", nat.KERNEL_KINDS), ("DIRAC_STEP_AUTO", nat.STEP_AUTO),
                        ("DIRAC_STEP_PASSES", nat.STEP_PASSES),
                        ("DIRAC_STEP_ONE_LAUNCH", nat.STEP_ONE_LAUNCH),
                        ("DIRAC_EIG_RITZ_MAX", nat.EIG_RITZ_MAX), ("DIRAC_EIG_ITER_MAX", nat.EIG_ITER_MAX)):
        assert int(defs[name]) == value, name


def test_calls_on_null_context_fail_cleanly(lib):
    assert lib.dirac_set_step_mode(None, 0) == nat.EINVAL
    assert lib.dirac_debug_barrier_timeout(None, None, 1e-4, 4) == nat.EINVAL
    assert lib.dirac_state_bytes(None) == 0
    assert lib.dirac_export_state(None, None, 0) == nat.EINVAL
    assert lib.dirac_import_state(None, None, 0) == nat.EINVAL
    assert lib.dirac_set_fields(None, None, 0.0, 0.0, 0.0) == nat.EINVAL
    assert lib.dirac_lanczos_step(None, None, 1e-4, 10, 0.0, None) == nat.EINVAL
    assert lib.dirac_sync(None) == nat.EINVAL
    lib.dirac_destroy(None)


def test_no_gpu_gives_cuda_error_not_a_crash(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = ctypes.c_void_p()
    st = lib.dirac_create(ctypes.byref(ctx), 8, 8, 0.1, 0.1, 1.0, 137.036, 2, 0, 0, 4, None)
    assert st in (nat.ECUDA, nat.ENOMEM)
    assert not ctx.value


def test_c99_client_compiles_links_and_runs(tmp_path, lib):
    """include/dirac.h is a C header: a C99 program (tests/c/abi_check.c)
    compiles against it with warnings as errors, links the library and gets
    the documented results from the calls that need no GPU."""
    import shutil
    import subprocess
    from paper_1407_7370_gb300 import build
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    so_dir = os.path.dirname(build.LIB)
    exe = str(tmp_path / "abi_check")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(build.ROOT, "include"), os.path.join(here, "c", "abi_check.c"),
           "-o", exe, "-L", so_dir, "-ldirac_gb300", "-Wl,-rpath," + so_dir, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and "abi_check ok" in run.stdout, run.stdout + run.stderr


@pytest.mark.gpu
def test_c99_client_propagates_on_the_gpu(tmp_path):
    """tests/c/propagate_check.c: device memory from the CUDA runtime, ten
    FP64 steps through the C ABI, unitary to 1e-12."""
    import shutil
    import subprocess
    from paper_1407_7370_gb300 import build
    build.build()
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    cuda = os.path.dirname(os.path.dirname(build.nvcc_path()))
    lib64 = next((p for p in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"),
                              os.path.join(cuda, "targets", "sbsa-linux", "lib"),
                              os.path.join(cuda, "targets", "x86_64-linux", "lib"))
                  if os.path.exists(os.path.join(p, "libcudart.so"))), None)
    if lib64 is None:
        pytest.fail("libcudart.so not found under " + cuda)
    here = os.path.dirname(os.path.abspath(__file__))
    so_dir = os.path.dirname(build.LIB)
    exe = str(tmp_path / "propagate_check")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(build.ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(here, "c", "propagate_check.c"), "-o", exe,
           "-L", so_dir, "-ldirac_gb300", "-Wl,-rpath," + so_dir, "-L", lib64, "-lcudart",
           "-Wl,-rpath," + lib64, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and "propagate_check ok" in run.stdout, run.stdout + run.stderr
