"""The measured FMA throughput (gks_fma_rate) that the benchmark divides
by: positive, below what GB300's FP64 and FP32 lanes can do at the highest
SM clock, and repeatable."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible_and_repeatable():
    import torch
    from paper_2508_19911_gb300 import gks
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    top = 2.2e9  # Hz, above GB300's highest SM clock (2.07 GHz)
    f64a, ms64 = gks.fma_rate("fp64")
    f64b, _ = gks.fma_rate("fp64")
    f32, ms32 = gks.fma_rate("fp32")
    # 2 FP64 and 128 FP32 FMA lanes per SM per clock, 2 FLOP per FMA
    assert 0.1 * sms * 4 * top < f64a < sms * 4 * top
    assert 0.1 * sms * 256 * top < f32 < sms * 256 * top
    assert abs(f64a - f64b) < 0.05 * f64a
    assert ms64 > 1.0 and ms32 > 1.0
