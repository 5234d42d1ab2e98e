"""The measured FP32 FMA throughput (imrp_fp32_peak), the roofline denominator
of the field kernel: plausible against the device's SM count (128 FP32 lanes
per SM, 2 flops per FMA, a clock of at most about 2.1 GHz) and stable."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp
    build.build()
    t1, sms = imrp.fp32_peak()
    t2, _ = imrp.fp32_peak()
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    per_sm_ghz = t1 * 1e3 / (sms * 128 * 2)  # implied clock in GHz at full issue
    print(f"FP32 peak {t1:.2f} / {t2:.2f} TFLOP/s on {sms} SMs ({per_sm_ghz:.3f} GHz at full FMA issue)")
    assert 0.8 < per_sm_ghz < 2.2
    assert abs(t1 - t2) < 0.1 * t1
