"""The FMA-pipe throughput measurement behind the arithmetic roofline of the
FP64-bound kernels (fv_fma_peak): both pipes give a rate in the range the
GPU's unit counts and clocks allow, and the FP32 pipe is the faster one."""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_fma_peak_rates_are_plausible():
    from paper_1701_05431_gb300 import fvlib
    stream = torch.cuda.current_stream().cuda_stream
    r64 = fvlib.fma_peak("f64", 0.01, stream)
    r32 = fvlib.fma_peak("f32", 0.01, stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clock_hz = 2.2e9                     # above any SM clock of the part
    assert 1e9 < r64 <= sms * 64 * clock_hz, r64
    assert 1e11 < r32 <= sms * 128 * clock_hz, r32
    assert r32 > 2 * r64
