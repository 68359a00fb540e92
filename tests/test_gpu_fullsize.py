"""Parity at the benchmark's full size (L = 4096, N = 1, 64 surfaces in uint64
words, 8x8 tiles, seed 0) on sampled outputs the oracle computes one lane at a
time: every height of lanes 0 and 63 and the exact sums of four lanes after a
few sweeps, through the same C-ABI calls and launch configuration bench.py
times."""
import numpy as np
import pytest

from rsos_testlib import assert_parity

pytestmark = pytest.mark.gpu


def test_ms_L4096_N1_S64_sampled_lanes():
    assert_parity(L=4096, N=1, S=64, T=8, seed=0, times=[0, 1, 3], t_end=3, lanes=[0, 31, 32, 63],
                  height_lanes=[0, 63], threads=4)
