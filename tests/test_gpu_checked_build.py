"""The bounds-checked build (RSOS_CHECKED): every record a sweep kernel
stages or writes back is tested against the lattice, and every shared-memory
record against the block's dynamic shared memory; failures are counted, not
trapped.  Jobs on every sweep engine must count zero and still match the
oracle bit for bit.  The checked library is built and loaded in a child
process (a process loads one librsos)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import sys
sys.path[:0] = [ROOT, HERE]
import numpy as np
import paper_1605_02620_gb300 as R
from rsos_testlib import oracle_run
assert R.rsos_checked_build()
cases = [  # (L, N, S, T, tiling, engine, t_end)
    (64, 1, 64, 8, 0, 2, 20), (32, 3, 96, 4, 0, 1, 15), (64, 1, 64, (6, 10), 1, 0, 20),
    (37, 2, 96, (4, 5), 1, 0, 12), (128, 4, 64, 16, 0, 2, 8), (64, 2, 2048, 8, 0, 1, 4),
]
for (L, N, S, T, tiling, engine, t_end) in cases:
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=T, seed=3, engine=engine, series_capacity=4, tiling=tiling)
    h = R.rsos_init(p)
    try:
        R.rsos_schedule(h, [t_end])
        R.rsos_sweep(h, t_end)
        ts, s1, s2, _ = R.rsos_read_series(h, S, 4)
        errors = R.rsos_bounds_errors(h)
    finally:
        R.rsos_free(h)
    assert errors == 0, (L, N, S, T, tiling, engine, errors)
    lanes = [0, S - 1]
    ots, o1, o2, _ = oracle_run(L, N, lanes, T, seed=3, times=[t_end], t_end=t_end, tiling=tiling)
    for c, j in enumerate(lanes):
        assert int(s1[0, j]) == int(o1[0, c]) and int(s2[0, j]) == int(o2[0, c]), (L, N, j)
print("checked ok", len(cases))
"""


def test_checked_build_counts_no_out_of_range_access():
    from paper_1605_02620_gb300 import build as B
    B.build(checked=True)
    env = dict(os.environ, RSOS_CHECKED="1")
    code = CHILD.replace("ROOT", repr(ROOT)).replace("HERE", repr(HERE))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked ok" in r.stdout
