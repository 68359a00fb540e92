"""Closed forms for N -> infinity, where Eq. 6 never rejects and RSOS growth
reduces to random deposition.

RS (one uniformly chosen site per attempt, L^2 attempts per step):
    h(x) ~ Binomial(t L^2, 1/L^2), sum h fixed  =>  E[W^2](t) = t (1 - 1/L^2).
DT (per sweep every sub-tile of a sites gets 2a selections, each a uniform
site with a fair mask bit):  per sweep a site receives Binomial(2a, 1/(2a))
deposits, sites of one sub-tile are multinomially anti-correlated
(covariance -1/(2a)), and the total is Binomial(2L^2, 1/2), so
    E[W^2](t) = t (1 - 1/(2a) - 1/(2 L^2)).
These pin the number of selections per activation (2a), the mask
probability (1/2) and the sub-tile size a = (Tx/2)(Ty/2).

Lanes of one job share the selected sites (section II), so they are not
independent samples: errors are taken across independent seeds.
"""
import math

import numpy as np
import pytest

import oracle as O

FREE = 10 ** 9


def _mean_w2(make, n_seeds, lanes, t, rs):
    per_seed, totals = [], []
    for seed in range(n_seeds):
        p = make(seed)
        h = O.flat(p.L, len(lanes))
        O.sweeps(p, h, lanes, 0, t, rs=rs)
        s1, s2 = O.sums(h)
        per_seed.append(np.mean([O.width2(a, b, p.L) for a, b in zip(s1, s2)]))
        totals.extend(s1)
    w2 = np.array(per_seed)
    return w2.mean(), w2.std(ddof=1) / math.sqrt(len(w2)), totals


@pytest.mark.parametrize("T", [8, 4])
def test_dt_random_deposition_width(T):
    L, t = 32, 40
    mean, err, _ = _mean_w2(lambda s: O.Params(L=L, N=FREE, Tx=T, Ty=T, seed=1000 + s), 64,
                            list(range(8)), t, rs=False)
    a = (T // 2) ** 2
    expect = t * (1 - 1 / (2 * a) - 1 / (2 * L * L))
    assert abs(mean - expect) < 4 * err, (mean, expect, err)
    # the RS value is excluded: distinguishes the sub-tile anti-correlation
    assert abs(mean - t * (1 - 1 / (L * L))) > 4 * err


def test_dt_total_deposits_are_binomial():
    # sum h after one sweep ~ Binomial(2 L^2, 1/2) per lane
    L = 32
    acc = []
    for seed in range(256):
        h = O.flat(L, 1)
        acc.append(O.sweeps(O.Params(L=L, N=FREE, seed=seed), h, [seed % 64], 0, 1)[0])
    acc = np.array(acc, dtype=float)
    n = 2 * L * L
    assert abs(acc.mean() - n / 2) < 4 * math.sqrt(n / 4 / 256)
    assert abs(acc.var(ddof=1) - n / 4) < 0.3 * n / 4


def test_rs_random_deposition_width():
    L, t = 32, 40
    mean, err, s1 = _mean_w2(lambda s: O.Params(L=L, N=FREE, seed=2000 + s), 48, [0, 1], t, rs=True)
    assert all(v == t * L * L for v in s1)
    expect = t * (1 - 1 / (L * L))
    assert abs(mean - expect) < 4 * err, (mean, expect, err)
