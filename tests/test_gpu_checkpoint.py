"""Checkpoint / resume: a job snapshotted at t1 and restored into a new handle
(here also through a file) continues bit-identically to the uninterrupted
job — sums, moments, heights and the measured series."""
import numpy as np
import pytest

import paper_1605_02620_gb300 as R

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,S,moments", [(256, 1, 64, False), (64, 1, 1, False), (128, 2, 32, True)])
def test_resume_is_bit_exact(L, N, S, moments, tmp_path):
    times = [0, 2, 5, 9, 14]
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=8, seed=99, series_capacity=8)

    def start():
        h = R.rsos_init(p)
        R.rsos_set_moments(h, moments)
        R.rsos_schedule(h, times)
        return h

    def finish(h):
        R.rsos_sweep(h, 14 - R.rsos_time(h))
        ts, sums, has = R.rsos_read_moments(h, S, 8)
        heights = [R.rsos_heights(h, j, L) for j in (0, S - 1)]
        R.rsos_free(h)
        return ts, sums, has, heights

    a = start()
    ref = finish(a)

    b = start()
    R.rsos_sweep(b, 7)
    snap = R.rsos_snapshot(b)
    assert len(snap) == R.rsos_snapshot_bytes(b)
    R.rsos_free(b)
    path = tmp_path / "job.rsos"
    path.write_bytes(snap)
    c = R.rsos_restore(path.read_bytes())
    assert R.rsos_time(c) == 7
    got = finish(c)

    assert list(got[0]) == list(ref[0]) == times
    assert (got[1] == ref[1]).all() and (got[2] == ref[2]).all()
    for x, y in zip(got[3], ref[3]):
        assert np.array_equal(x, y)
