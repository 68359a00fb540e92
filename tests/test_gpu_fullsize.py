"""Parity at full size, on sampled outputs the oracle computes one lane at a
time, through the same C-ABI calls and launch configuration bench.py times:
the benchmark workload (L = 4096, N = 1, 64 surfaces in uint64 words, 8x8
tiles, seed 0: every height of lanes 0 and 63 and the exact sums of four
lanes after a few sweeps) and the step-height workload (L = 32768, 32
surfaces, N = 1 and 4: the exact sums of one lane after one sweep)."""
import numpy as np
import pytest

from rsos_testlib import assert_parity

pytestmark = pytest.mark.gpu


def test_ms_L4096_N1_S64_sampled_lanes():
    assert_parity(L=4096, N=1, S=64, T=8, seed=0, times=[0, 1, 3], t_end=3, lanes=[0, 31, 32, 63],
                  height_lanes=[0, 63], threads=4)


@pytest.mark.parametrize("N", [1, 4])
def test_step_height_L32768_S32_sampled_lane(N):
    # Step-height workload at full size (8 / 16 GiB of planes): the exact sums
    # of lane 31 after one sweep (the oracle runs that lane alone).
    assert_parity(L=32768, N=N, S=32, T=8, seed=0, times=[0, 1], t_end=1, lanes=[31], height_lanes=[], threads=1)
