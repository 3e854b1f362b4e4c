"""The device-rate probes behind the roofline denominators (sim_measure_peak).

Each kind returns a positive rate in a plausible range for one GB300-class
GPU, and an unknown kind is rejected with SIM_EINVAL.  The ranges are wide:
they catch a probe that times nothing (or the wrong number of bytes or
flops), not small run-to-run differences.
"""
import pytest

import paper_2303_00689_gb300 as kx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def test_rates_are_plausible():
    fp64 = kx.sim_measure_peak(0)
    fp32 = kx.sim_measure_peak(1)
    l2 = kx.sim_measure_peak(2)
    print(f"FP64 {fp64:.2f} TFLOP/s, FP32 {fp32:.1f} TFLOP/s, L2 read+write {l2:.2f} TB/s")
    assert 0.1 < fp64 < 50.0
    assert 10.0 < fp32 < 500.0
    assert fp32 > 10.0 * fp64
    assert 1.0 < l2 < 100.0


def test_unknown_kind_is_rejected():
    with pytest.raises(kx.SimError) as e:
        kx.sim_measure_peak(3)
    assert e.value.code == kx.SIM_EINVAL
