"""The oracle's (+1) tilings (section III.C: domains of 6(+1) x 10(+1) sites)
pinned to what the paper and the mathematics fix.

* With T even and dividing L a (+1) tiling is the regular tiling of section
  II, so both sweeps must give the same heights, bit for bit; so is a single
  (T + 1)-wide tile per axis on L = T + 1, reached through the (+1) rule.
* The halves of every axis partition the lattice and the halves of one set
  never touch, which is what lets a set be updated in parallel (section II).
* N -> infinity (random deposition): a site of a sub-tile of a sites receives
  Binomial(2a, 1/(2a)) deposits per sweep, sites of one sub-tile have
  covariance -1/(2a), and the total is Binomial(2 L^2, 1/2); summing over
  sites, every sub-tile contributes 1/2 to sum_x 1/(2 a_x), so
      E[W^2](t) = t (1 - n_sub / (2 L^2) - 1 / (2 L^2))
  with n_sub = 4 (L div Tx)(L div Ty) sub-tiles per sweep (the regular
  formula t (1 - 1/(2a) - 1/(2L^2)) when n_sub = L^2 / a).  A selection picks
  k = floor(u a / 2^16) from a 16-bit u, uniform to within a / 2^16 when a
  is not a power of two: far below the tolerance here.
* Long runs on L = 3 (one 3-site tile per axis, halved into 1 + 2 sites)
  reproduce the exact stationary velocity and width of the chain enumerated
  by ``oracle/enumerate.py`` (tests/golden/enumeration.json, section
  dt_general).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

FREE = 10 ** 9
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "enumeration.json")


@pytest.mark.parametrize("L,N,Tx,Ty,order", [
    (16, 1, 4, 4, 0), (24, 2, 8, 4, 0), (32, 3, 8, 8, 1), (12, 1, 2, 6, 0), (16, 7, 16, 8, 0),
])
def test_reduces_to_regular_tiling(L, N, Tx, Ty, order):
    lanes = [0, 5, 37, 63]
    a = O.flat(L, len(lanes))
    b = O.flat(L, len(lanes))
    O.sweeps(O.Params(L=L, N=N, Tx=Tx, Ty=Ty, phase_order=order, seed=L + N), a, lanes, 0, 25)
    O.sweeps(O.Params(L=L, N=N, Tx=Tx, Ty=Ty, phase_order=order, seed=L + N, tiling=1), b, lanes, 0, 25)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("L,T", [(64, 6), (64, 10), (9605, 6), (9605, 10), (9605, 8), (3, 2), (5, 2),
                                 (37, 5), (50, 8), (27, 3), (130, 13), (7, 3)])
def test_halves_partition_the_axis(L, T):
    n, r = L // T, L % T
    assert r <= n
    spans = []
    for c in range(n):
        (s0, w0), (s1, w1) = O.axis_half(L, T, c, 0), O.axis_half(L, T, c, 1)
        assert w0 >= 1 and w1 >= 1 and w0 <= w1 <= w0 + 1
        assert w0 + w1 == (T + 1 if c < r else T)
        spans += [(s0, w0, 0), (s1, w1, 1)]
    # consecutive, covering [0, L) exactly once, alternating halves
    x = 0
    for s, w, half in spans:
        assert s == x
        x += w
    assert x == L
    assert [h for _, _, h in spans] == [0, 1] * n
    # two halves of the same set are separated by at least one site of the
    # other set (periodically), so parallel updates never touch
    for c in range(n):
        for half in (0, 1):
            s, w = O.axis_half(L, T, c, half)
            nxt = O.axis_half(L, T, (c + 1) % n, half)[0] + (L if c == n - 1 else 0)
            assert nxt - (s + w) >= 1


def test_origin_covers_one_period():
    # irregular axis: the pattern repeats only after L sites; regular: after T
    p = O.Params(L=64, N=1, Tx=6, Ty=8, seed=11, tiling=1)
    xs, ys = zip(*[O.control(p, t)[:2] for t in range(4000)])
    assert min(xs) == 0 and max(xs) == 63 and len(set(xs)) == 64
    assert min(ys) == 0 and max(ys) == 7 and len(set(ys)) == 8


def _rd_width(L, Tx, Ty, t, n_seeds, lanes):
    per_seed, totals = [], []
    for seed in range(n_seeds):
        p = O.Params(L=L, N=FREE, Tx=Tx, Ty=Ty, seed=3000 + seed, tiling=1)
        h = O.flat(L, len(lanes))
        O.sweeps(p, h, lanes, 0, t)
        s1, s2 = O.sums(h)
        per_seed.append(np.mean([O.width2(a, b, L) for a, b in zip(s1, s2)]))
        totals.extend(s1)
    w2 = np.array(per_seed)
    return w2.mean(), w2.std(ddof=1) / math.sqrt(len(w2)), np.array(totals, dtype=float)


@pytest.mark.parametrize("L,Tx,Ty", [(64, 6, 10), (37, 4, 5)])
def test_random_deposition_width(L, Tx, Ty):
    t, lanes = 40, list(range(8))
    mean, err, totals = _rd_width(L, Tx, Ty, t, 64, lanes)
    n_sub = 4 * (L // Tx) * (L // Ty)
    expect = t * (1 - n_sub / (2 * L * L) - 1 / (2 * L * L))
    assert abs(mean - expect) < 4 * err, (mean, expect, err)
    # every sub-tile of a sites gets 2a selections with a fair mask bit:
    # total deposits ~ Binomial(2 L^2 t, 1/2) per lane
    n = 2 * L * L * t
    assert abs(totals.mean() - n / 2) < 4 * math.sqrt(n / 4 / totals.size)


def _golden_general():
    with open(GOLDEN) as f:
        return json.load(f)["dt_general"]


@pytest.mark.parametrize("case", _golden_general(),
                         ids=lambda c: f"L{c['L']}-N{c['N']}-T{c['Tx']}x{c['Ty']}-o{c['phase_order']}")
def test_long_runs_match_exact_chain(case):
    L, N = case["L"], case["N"]
    v_seed, w_seed = [], []
    burn, blocks, block_len = 300, 40, 50
    for seed in range(16):
        p = O.Params(L=L, N=N, Tx=case["Tx"], Ty=case["Ty"], phase_order=case["phase_order"],
                     seed=7919 * seed + 17, tiling=1)
        lanes = list(range(8))
        h = O.flat(L, len(lanes))
        O.sweeps(p, h, lanes, 0, burn)
        s_start, _ = O.sums(h)
        t, w2 = burn, []
        for _ in range(blocks):
            O.sweeps(p, h, lanes, t, block_len)
            t += block_len
            s1, s2 = O.sums(h)
            w2.append(np.mean([O.width2(a, b, L) for a, b in zip(s1, s2)]))
        s_end, _ = O.sums(h)
        v_seed.append(np.mean([(b - a) / (L * L * (t - burn)) for a, b in zip(s_start, s_end)]))
        w_seed.append(np.mean(w2))
    v, w = np.array(v_seed), np.array(w_seed)
    dv, dw = v.std(ddof=1) / math.sqrt(len(v)), w.std(ddof=1) / math.sqrt(len(w))
    assert abs(v.mean() - case["velocity"]) < 4.5 * dv + 1e-9, (v.mean(), dv, case["velocity"])
    assert abs(w.mean() - case["w2"]) < 4.5 * dw + 1e-9, (w.mean(), dw, case["w2"])
    # the (+1) chain differs from the regular L = 2 chain and from RS at L = 3
    # by far more than the error: the test sees the tiling
    assert abs(case["velocity"] - 0.39422098080284623) > 10 * dv or N != 1


def test_rejects_impossible_tilings():
    h = O.flat(10, 1)
    with pytest.raises(ValueError):  # 10 = 1 x 7 + 3: three extra sites for one tile
        O.sweeps(O.Params(L=10, N=1, Tx=7, Ty=2, tiling=1), h, [0], 0, 1)
    with pytest.raises(ValueError):  # sub-tiles need at least one site
        O.sweeps(O.Params(L=10, N=1, Tx=1, Ty=2, tiling=1), h, [0], 0, 1)


@pytest.mark.parametrize("L,N", [(4, 1), (6, 2), (8, 3)])
def test_single_wide_tile_is_the_regular_tiling(L, N):
    """L = T + 1 with T + 1 even: one tile of L sites per axis, halved into
    L/2 + L/2, and the origin uniform over L — the regular tiling with edge L,
    reached through the (+1) rule (r = 1), bit for bit."""
    lanes = [0, 9, 33]
    a = O.flat(L, len(lanes))
    b = O.flat(L, len(lanes))
    O.sweeps(O.Params(L=L, N=N, Tx=L, Ty=L, seed=L), a, lanes, 0, 40)
    O.sweeps(O.Params(L=L, N=N, Tx=L - 1, Ty=L - 1, seed=L, tiling=1), b, lanes, 0, 40)
    assert np.array_equal(a, b)
