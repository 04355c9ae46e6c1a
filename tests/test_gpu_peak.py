"""The measured FMA peaks the roofline divides by (lj_measure_peak) are
plausible: positive, below the issue limit of the device's FP32 lanes at
2.2 GHz (no GB300 clock is higher), and FP64 far below FP32 on GB300."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import torch
    from paper_0709_3225_gb300 import lj
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32, ms32, sms = lj.lj_measure_peak(lj.PEAK_FP32)
    fp32x2, _, _ = lj.lj_measure_peak(lj.PEAK_FP32X2)
    fp64, ms64, _ = lj.lj_measure_peak(lj.PEAK_FP64)
    assert sms == nsm
    assert ms32 >= 20.0 and ms64 >= 20.0
    limit32 = nsm * 128 * 2 * 2.2e9
    for v in (fp32, fp32x2):
        assert 0.2 * limit32 < v <= limit32
    assert 0.0 < fp64 < 0.2 * fp32
    with pytest.raises(lj.LJError):
        lj.lj_measure_peak(3)
