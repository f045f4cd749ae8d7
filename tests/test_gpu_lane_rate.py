"""vdwdf_lane_rate, the measured denominators of the pair kernels' ALU rooflines:
the FP32 FMA rate must sit near the unit-count peak (SMs x 128 FP32 lanes x the
SM clock, at most 2070 MHz on GB300), FP64 below FP32, each call launches
two to four kernels (a calibration and the sized timed launches), and the
timed launch lasts at least half of what was asked."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    import paper_0810_2273_gb300 as V
    return V


def test_lane_rates(V):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    unit_peak = sms * 128 * 2070e6          # FP32 lane operations/s at the maximum SM clock
    rates = {}
    for kind in ("fp32", "fp32x2", "fp64"):
        l0 = V.launch_count()
        r, ms = V.lane_rate(kind, 20.0)
        assert 2 <= V.launch_count() - l0 <= 4, kind
        assert r > 0.0 and 10.0 <= ms < 200.0, (kind, r, ms)
        rates[kind] = r
    # the FP32 pipe: 128 lanes per SM; more than the unit count would mean the
    # kernel did less work than it counts, far less that it is not pipe-bound
    assert 0.5 * unit_peak < rates["fp32"] <= 1.02 * unit_peak, rates["fp32"] / unit_peak
    assert 0.5 * unit_peak < rates["fp32x2"] <= 2.04 * unit_peak, rates["fp32x2"] / unit_peak
    assert rates["fp64"] < rates["fp32"]


def test_lane_rate_refusals(V):
    with pytest.raises(ValueError):
        V.lane_rate("int8")
    with pytest.raises(V.VdwdfError):
        V.lane_rate("fp32", 0.1)
