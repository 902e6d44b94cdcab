"""The FMA-throughput diagnostic the bench quotes beside its FP64 rooflines."""
import pytest

from paper_1311_4627_gb300 import heat

pytestmark = pytest.mark.gpu


def test_measured_fma_peaks():
    """The roofline diagnostic: FP64 FMA throughput near the nominal 1.25 TFLOP/s of a GB300
    (1/64 of the FP32 rate), and FP32 about 64 times faster."""
    f64 = heat.heat_measure_fma_peak(0, True)
    f32 = heat.heat_measure_fma_peak(0, False)
    assert 0.8 < f64 < 1.4, f64
    assert 30.0 < f32 / f64 < 100.0, (f32, f64)
