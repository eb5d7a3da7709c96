"""The FMA-rate microbenchmark behind the FP64 path's arithmetic roofline:
it runs, reports a positive rate, FP32 above FP64 (GB300's FP64 rate is a
small fraction of its FP32 rate), and the FP32 rate not above the CUDA
cores' nominal peak (152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.6
TFLOP/s, with 10% allowance for the clock)."""
import pytest

from _helpers import gpu

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible():
    lm = gpu()
    f64 = lm.sw_fma_peak("f64", 1024)
    f32 = lm.sw_fma_peak("f32", 1024)
    assert 0.0 < f64 < f32
    assert f32 < 80.6 * 1.1
