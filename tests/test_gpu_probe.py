"""gpe_probe_peak: the measured multiply-add rates behind the roofline of the
operator kernels (float32, packed float32, float64)."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402


def test_probe_rates_are_plausible():
    f32 = G.probe_peak(0)
    f32x2 = G.probe_peak(1)
    f64 = G.probe_peak(2)
    for v in (f32, f32x2, f64):
        assert math.isfinite(v) and v > 0.0
    # a GB300-class part: tens of TFLOP/s in float32, float64 well below it
    assert 10.0 < f32 < 500.0
    assert f32x2 > 0.5 * f32
    assert f64 < f32
    print(f"float32 FMA {f32:.1f} TFLOP/s, packed float32 {f32x2:.1f}, float64 {f64:.2f}")


def test_probe_rejects_unknown_kind():
    with pytest.raises(G.GPEError):
        G.probe_peak(7)
