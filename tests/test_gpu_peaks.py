"""The integer-throughput probes behind the integer-pipe roofline: rates are
positive, below the nominal lane counts of the GPU (152 SMs x 128 lanes x the
maximum SM clock), and far from zero (a probe whose chain was optimised away
would report an impossible rate)."""
import pytest

import paper_1605_02620_gb300 as R

pytestmark = pytest.mark.gpu

NOMINAL_LANE_OPS = 152 * 128 * 2.07e9  # every lane of every SM each clock


@pytest.mark.parametrize("kind", [0, 1])
def test_int_probe_rates_are_physical(kind):
    r = R.rsos_peak_int(kind, 4096)
    assert 0.1 * NOMINAL_LANE_OPS < r < 1.05 * NOMINAL_LANE_OPS, r


def test_philox_probe_rate_is_physical():
    # a Philox-4x32-10 block is at least 10 rounds of 2 multiplies
    r = R.rsos_peak_int(2, 512)
    assert 1e9 < r < NOMINAL_LANE_OPS / 20, r
