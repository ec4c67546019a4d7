"""hweno_fma_peak, the measured denominator of the stage kernels' arithmetic
roofline: FP32 and FP64 FMA throughput of the device."""

import pytest

from paper_2002_08816_gb300 import hweno as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def test_fma_peak_is_plausible():
    """The FP32 rate is a few tens of TFLOP/s on a GPU of this class and no
    more than 2 flops x 128 lanes x the SMs x 2.5 GHz; FP64 is far below it."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = H.hweno_fma_peak(False, 2000)
    f64 = H.hweno_fma_peak(True, 100)
    assert 1e12 < f32 <= 2 * 128 * sms * 2.5e9
    assert 0 < f64 < f32
    # packed FP32 (two FMAs per instruction) within the same lane-rate bound
    f32x2 = H.hweno_fma_peak(2, 1000)
    assert 1e12 < f32x2 <= 2 * 128 * sms * 2.5e9
