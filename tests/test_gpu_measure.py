"""The FMA-chain kernels that check the fused step's derived ALU peak
(ag_measure_fp32_peak): launch shape, and that the reported rates follow
from the work done and the measured times."""
import pytest
import torch

from paper_2305_16510_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def test_fp32_peak_rates_follow_from_work_and_time():
    r = _abi.ag_measure_fp32_peak(torch.cuda.current_stream().cuda_stream, iters=2000, reps=3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert r["block"] == 256 and r["grid"] % sms == 0 and r["grid"] >= sms
    fma = r["grid"] * r["block"] * 8 * 16 * 2000          # chains x rounds x iters per thread
    assert r["scalar_ms"] > 0 and r["packed_ms"] > 0
    assert r["scalar_tflops"] == pytest.approx(2 * fma / (r["scalar_ms"] * 1e-3) / 1e12, rel=1e-9)
    assert r["packed_tflops"] == pytest.approx(4 * fma / (r["packed_ms"] * 1e-3) / 1e12, rel=1e-9)
    # no device does more than 128 FP32 FMAs per SM per clock at 3 GHz
    bound = sms * 128 * 2 * 3.0e9 / 1e12
    assert 0 < r["scalar_tflops"] < bound and 0 < r["packed_tflops"] < bound
