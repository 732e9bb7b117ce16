"""The FMA-rate probe (tl_probe_fma_rates) on the GPU: positive rates, FP32
far above FP64 on this part, FP64 not above 2 FMA per clock per SM (the
pipe's width here) at any plausible clock."""
import pytest
import torch

from paper_2607_24908_gb300 import tl as T

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    f64, f32 = T.tl_probe_fma_rates()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert f64 > 0 and f32 > 0
    assert f32 > 8 * f64
    assert f64 < 2 * sms * 2.3e9
    assert f32 < 128 * sms * 2.3e9
