"""The FP32 rate microbenchmark behind the P2P roofline (fmm_measure_fp32_rate)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_rate_is_plausible():
    import torch

    from paper_1206_0115_b300 import fmm
    r = fmm.fmm_measure_fp32_rate()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert int(r[2]) == sms
    # 128 FP32 lanes per SM, 2 flop per FMA: the measured rate lies below
    # lanes x 2 x a 2.1 GHz ceiling and above a third of it at 1 GHz
    ceiling = sms * 128 * 2 * 2.1e9
    for rate in r[:2]:
        assert ceiling / 6 < rate < ceiling
