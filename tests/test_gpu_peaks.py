"""The arithmetic peak probe that supplies the Legendre stages' roofline
denominators returns plausible rates on a GB300: the FP32 pipe's scalar and
packed FMA rates near the 152 SM x 128 lane x 2 flop x clock figure (80.5
TFLOP/s at 2070 MHz; the clock under load may be lower), and the FP64 rate
near the part's nominal 1.25 TFLOP/s."""
import pytest

from gpu_util import cuda_device
from paper_1308_5299_gb300 import binding

pytestmark = pytest.mark.gpu


def test_fma_peaks_plausible():
    cuda_device()
    f32 = binding.fma_peak("f32")
    f32x2 = binding.fma_peak("f32x2")
    f64 = binding.fma_peak("f64")
    print("FMA peaks (TFLOP/s): f32 %.2f, f32x2 %.2f, f64 %.3f" % (f32, f32x2, f64))
    assert 40.0 < f32 < 90.0
    assert 0.8 * f32 < f32x2 < 2.2 * f32
    assert 0.5 < f64 < 3.0
