"""The measured arithmetic peak (dirac_measure_peak), the denominator of the
roofline of the FP64 path: plausible against the GB300's unit counts (152
SMs, two FP64 and 128 FP32 fused multiply-adds per clock per SM, at most
2.07 GHz) -- at most the nominal figure, and at least a third of it."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_1407_7370_gb300 import build
    from paper_1407_7370_gb300 import _native
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return _native


@pytest.mark.parametrize("kind,per_clk", [(0, 2), (1, 128)])
def test_measured_fma_peak_is_plausible(nat, kind, per_clk):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * per_clk * 2 * 2.07e9 / 1e12   # TFLOP/s at the highest SM clock
    t = ctypes.c_double(0.0)
    nat.check(nat.lib().dirac_measure_peak(kind, ctypes.byref(t)))
    assert nominal / 3.0 <= t.value <= nominal * 1.02, (kind, t.value, nominal)


def test_measure_peak_rejects_unknown_kinds(nat):
    t = ctypes.c_double(0.0)
    assert nat.lib().dirac_measure_peak(7, ctypes.byref(t)) == nat.EINVAL
