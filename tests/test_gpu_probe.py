"""The FMA peak probes (hdf_probe_peaks) give the FP32 and FP64 rates that the
benchmark's roofline fractions divide by: both positive, FP32 within a factor
of two of the nominal unit count x clock figure (152 SMs x 128 lanes x 2 x
2.07 GHz = 80.5 TFLOP/s), FP64 far below FP32 on this part."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_probe_peaks_are_plausible():
    from paper_1811_02363_gb300 import build
    build.build()
    from paper_1811_02363_gb300 import api
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32, fp64 = api.probe_peaks()
    nominal = sms * 128 * 2 * 2.07e9 / 1e12
    print(f"FP32 {fp32:.1f} TFLOP/s (nominal {nominal:.1f}), FP64 {fp64:.2f} TFLOP/s")
    assert 0.5 * nominal <= fp32 <= 1.2 * nominal
    assert 0.0 < fp64 < fp32
