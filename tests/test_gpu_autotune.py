"""The autotuner of the execution geometry: what it picks is a valid geometry
that reproduces the untuned job bit for bit, it is cached per job shape, and
jobs outside the persistent engine come back unchanged."""
import time

import numpy as np
import pytest

import paper_1605_02620_gb300 as R
from rsos_testlib import gpu_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,S", [(256, 1, 64), (512, 2, 64), (256, 4, 32)])
def test_tuned_geometry_is_exact_and_cached(L, N, S):
    base = R.rsos_params(L=L, N=N, surfaces=S, tile=8, seed=5, series_capacity=8)
    tuned, us = R.rsos_autotune(base, sweeps=5)
    assert us > 0
    assert tuned.words_per_thread in (1, 2) and tuned.tiles_per_lane >= 1 and tuned.phase_lag in (0,) + tuple(
        range(2, L))
    assert (tuned.L, tuned.N, tuned.surfaces, tuned.tile_x, tuned.seed) == (L, N, S, 8, 5)
    t0 = time.perf_counter()
    again, us2 = R.rsos_autotune(base, sweeps=5)
    assert time.perf_counter() - t0 < 0.05 and us2 == us
    assert (again.words_per_thread, again.tiles_per_lane, again.phase_lag) == (
        tuned.words_per_thread, tuned.tiles_per_lane, tuned.phase_lag)
    # the tuned geometry gives the same job, bit for bit
    kw = dict(L=L, N=N, S=S, T=8, seed=5, times=[0, 3, 9], t_end=9, height_lanes=[0, S - 1])
    a = gpu_run(**kw)
    p = tuned
    h = R.rsos_init(p)
    try:
        R.rsos_schedule(h, kw["times"])
        R.rsos_sweep(h, kw["t_end"])
        ts, s1, s2, _ = R.rsos_read_series(h, S, 8)
        heights = {j: R.rsos_heights(h, j, L) for j in kw["height_lanes"]}
    finally:
        R.rsos_free(h)
    assert list(ts) == list(a[0]) and (s1 == a[1]).all() and (s2 == a[2]).all()
    for j in kw["height_lanes"]:
        assert np.array_equal(heights[j], a[4][j])


def test_jobs_outside_the_persistent_engine_unchanged():
    for p in (R.rsos_params(L=64, N=1, surfaces=1, tile=8, seed=1),  # plain path
              R.rsos_params(L=32, N=1, surfaces=64, tile=8, seed=1)):  # 4 tile rows: phase engine
        tuned, us = R.rsos_autotune(p, sweeps=3)
        assert (tuned.words_per_thread, tuned.tiles_per_lane, tuned.phase_lag) == (0, 0, 0) and us == 0.0
