"""The FMA-rate probe that gives the FP64 form its arithmetic ceiling.

Bounds, not values: the probe must report a positive rate between a tenth
and ten times the nominal per-GPU FMA throughput of a GB300 (FP64 about
1.2 TFLOP/s, FP32 152 SMs x 128 lanes x 2 FLOP x ~2 GHz = 78 TFLOP/s), and
FP32 must run well above FP64 on this part."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clbm():
    from paper_1908_05396_gb300 import build
    build.build()
    from paper_1908_05396_gb300 import clbm as c
    c.lib()
    return c


def test_probe_rates_are_plausible(clbm):
    f64 = clbm.probe_fma_rate("f64")
    f32 = clbm.probe_fma_rate("f32")
    assert 0.12e12 <= f64 <= 12e12
    assert 7.8e12 <= f32 <= 780e12
    assert f32 > 8 * f64
    with pytest.raises(clbm.CLBMError):
        clbm.probe_fma_rate("f16s")
