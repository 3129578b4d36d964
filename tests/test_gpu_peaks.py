"""sar_alu_peaks: measured FP32 and MUFU pipe throughput, the cross-check of the
backprojection's ALU roofline (nominal: 128 FP32 lanes and 16 MUFU lanes per
SM per clock)."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible():
    import torch
    import paper_2306_09784_gb300 as sar
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p = sar.alu_peaks()
    # no part of this family clocks above 2.2 GHz or below 0.5 GHz under load
    for key, lanes in (("fma_lane_ops_per_s", 128), ("ffma2_lane_ops_per_s", 128),
                       ("mufu_ops_per_s", 16)):
        assert 0.5e9 * sms * lanes * 0.5 < p[key] < 2.2e9 * sms * lanes * 1.1, (key, p[key])
