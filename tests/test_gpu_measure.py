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


def test_alu_peak_query_reads_the_device():
    """ag_query_alu_peak: the SM count torch sees, the FP32 lanes of a
    Blackwell SM, a peak clock in the GHz range, the peak as their product,
    and the FMA-chain kernels reaching between 90 % and 102 % of it."""
    dev = torch.cuda.current_device()
    q = _abi.ag_query_alu_peak(dev)
    props = torch.cuda.get_device_properties(dev)
    assert q["sm_count"] == props.multi_processor_count
    assert (q["cc_major"], q["cc_minor"]) == (props.major, props.minor)
    if props.major == 10:
        assert q["fp32_lanes_per_sm"] == 128
    assert 1.0e6 < q["max_sm_clock_khz"] < 3.5e6
    derived = q["sm_count"] * q["fp32_lanes_per_sm"] * 2 * q["max_sm_clock_khz"] * 1e3 / 1e12
    assert q["tflops"] == pytest.approx(derived, rel=1e-12)
    r = _abi.ag_measure_fp32_peak(torch.cuda.current_stream().cuda_stream, iters=5000, reps=3)
    assert 0.9 * q["tflops"] < r["packed_tflops"] < 1.02 * q["tflops"]


def test_measurement_entry_points_reject_null_outputs():
    import ctypes
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(64, n_obstacles=2)
    fl.reset(None, 1)
    lib = _abi.lib()
    assert lib.ag_collision_tests_run(fl.ctx, None) == _abi.AG_ERR_INVALID
    assert lib.ag_depth_live_pairs(fl.ctx, 32, 24, ctypes.c_float(1.0), ctypes.c_float(10.0), None, None, 4,
                                   None) == _abi.AG_ERR_INVALID
    assert lib.ag_query_alu_peak(0, None) == _abi.AG_ERR_INVALID
    assert _abi.ag_collision_tests_run(fl.ctx) == 0           # nothing stepped yet
    fl.step(3)
    assert _abi.ag_collision_tests_run(fl.ctx) >= 64          # the first step tests every environment
    fl.close()
