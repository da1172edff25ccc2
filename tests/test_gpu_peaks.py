"""The measured peak rates (psq_measure_peaks) that the FP64 rooflines divide by: plausible for
a GB300 (FP64 about 1/64 of the FP32 FMA rate, nominal 1.25 TFLOP/s; FP32 about 152 SMs x
128 lanes x 2 FLOPs x 2 GHz; the SFU a quarter of the FP32 lanes) and repeatable."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import paper_2510_15204_gb300 as P
    a = P.measure_peaks()
    b = P.measure_peaks()
    print(a, b)
    assert 0.6 < a["fp64_tflops"] < 2.5, a
    assert 30.0 < a["fp32_tflops"] < 120.0, a
    assert 1000.0 < a["sfu_gops"] < 12000.0, a
    assert a["fp32_tflops"] > 16 * a["fp64_tflops"], a
    for k in a:
        assert abs(a[k] - b[k]) < 0.1 * a[k], (k, a[k], b[k])
