"""The measured FMA throughput used as the roofline denominator of the FFT kernels."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    f32 = ll.fma_peak("fp32")
    f64 = ll.fma_peak("fp64")
    # GB300: 152 SMs x 128 FP32 lanes x 2 flops x ~2 GHz ~ 80 TFLOP/s; FP64 is a small fraction
    assert 20.0 < f32 < 120.0
    assert 0.05 < f64 < f32
    with pytest.raises(ll.LLError):
        ll._check(ll._lib.ll_fma_peak(7, None, None))
