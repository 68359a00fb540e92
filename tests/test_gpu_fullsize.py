"""Parity at full size, through the same C-ABI calls and the same launch
configuration bench.py times (the persistent engine, 200-sweep launches),
against the oracle run on the host cores:

* the benchmark workload (L = 4096, N = 1, 64 surfaces in uint64 words, 8x8
  tiles, seed 0): every height of all 64 lanes after 100 sweeps, and every
  height of lanes 0, 31 and 63 after 1000 sweeps (five 200-sweep launches),
  with the exact sums of those lanes at every 200th sweep;
* the step-height workload (L = 32768, 32 surfaces, N = 1, 2, 4; 8, 12 and
  16 GiB of planes): the exact sums and every height of lanes 0 and 31 after
  10 sweeps.

The oracle is the bottleneck (about 10^11 attempts), so these are marked
slow; lane 0's sums at all 40 times up to 10^4 sweeps are out of reach of
the host within a test (about 1.7 10^11 attempts for that one lane)."""
import numpy as np
import pytest

import oracle as O
import paper_1605_02620_gb300 as R

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def gpu_job(L, N, S, seed=0):
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=8, seed=seed, series_capacity=16)
    return R.rsos_init(p)


def assert_lanes_equal(h, oracle_fields, lanes, L, S, what):
    s1, s2, _, _ = R.rsos_width(h, S)
    o1, o2 = O.sums(oracle_fields)
    for c, j in enumerate(lanes):
        assert int(s1[j]) == o1[c] and int(s2[j]) == o2[c], f"{what}: sums of lane {j}"
        assert np.array_equal(R.rsos_heights(h, j, L), oracle_fields[c]), f"{what}: heights of lane {j}"


def test_ms_L4096_N1_S64_all_lanes_100_sweeps():
    L, N, S = 4096, 1, 64
    lanes = list(range(S))
    h = gpu_job(L, N, S)
    try:
        R.rsos_sweep(h, 100)  # one persistent launch of 100 sweeps
        f = O.flat(L, S)
        O.sweeps(O.Params(L=L, N=N, Tx=8, Ty=8, seed=0), f, lanes, 0, 100)
        assert_lanes_equal(h, f, lanes, L, S, "t=100")
    finally:
        R.rsos_free(h)


def test_ms_L4096_N1_S64_lanes_0_31_63_1000_sweeps():
    L, N, S = 4096, 1, 64
    lanes = [0, 31, 63]
    p = O.Params(L=L, N=N, Tx=8, Ty=8, seed=0)
    h = gpu_job(L, N, S)
    f = O.flat(L, len(lanes))
    try:
        for k in range(5):
            R.rsos_sweep(h, 200)  # the launch bench.py times: 200 sweeps per persistent launch
            O.sweeps(p, f, lanes, 200 * k, 200)
            s1, s2, _, t = R.rsos_width(h, S)
            assert t == 200 * (k + 1)
            o1, o2 = O.sums(f)
            for c, j in enumerate(lanes):
                assert int(s1[j]) == o1[c] and int(s2[j]) == o2[c], (t, j)
        for c, j in enumerate(lanes):
            assert np.array_equal(R.rsos_heights(h, j, L), f[c]), f"heights of lane {j} at t=1000"
    finally:
        R.rsos_free(h)


@pytest.mark.parametrize("N", [1, 2, 4])
def test_step_height_L32768_S32_lanes_0_31_10_sweeps(N):
    L, S = 32768, 32
    lanes = [0, 31]
    h = gpu_job(L, N, S)
    try:
        R.rsos_sweep(h, 10)
        f = O.flat(L, len(lanes))
        O.sweeps(O.Params(L=L, N=N, Tx=8, Ty=8, seed=0), f, lanes, 0, 10)
        assert_lanes_equal(h, f, lanes, L, S, f"N={N} t=10")
    finally:
        R.rsos_free(h)
