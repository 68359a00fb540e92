"""Statistical checks of the CUDA path against exact results and against the
paper's exponents (section III).  Seeds are fixed, so the outcomes are
deterministic; tolerances are several standard errors wide.

* Tiny lattices: the GPU's DT dynamics reproduces the exact stationary growth
  velocity and squared width of the enumerated Markov chains.
* Growth regime (Eq. 9): the effective exponent beta_eff of W(t) for N = 1
  at L = 4096 lies near the paper's beta = 0.241(1) (Table I; early times
  carry corrections, so the band is wide).
* Steady state (Eq. 12): the saturated width over L = 32..256 scales with an
  exponent near alpha = 0.390(4) (the paper's direct fits over 32 <= L <= 512
  give 0.392(1) for N = 1).
"""
import json
import math
import os

import numpy as np
import pytest

import paper_1605_02620_gb300 as R

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "enumeration.json")


def _series(L, N, S, seed, times, T=8, order=0):
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=T, phase_order=order, seed=seed,
                      series_capacity=len(times) + 2)
    h = R.rsos_init(p)
    try:
        R.rsos_schedule(h, times)
        R.rsos_sweep(h, times[-1])
        return R.rsos_read_series(h, S, len(times) + 2)
    finally:
        R.rsos_free(h)


@pytest.mark.parametrize("L,N,T,order", [(2, 1, 2, 0), (2, 2, 2, 0), (4, 1, 2, 1), (4, 1, 4, 1), (4, 1, 2, 0)])
def test_dt_dynamics_matches_exact_chain(L, N, T, order):
    g = json.load(open(GOLDEN))
    case = next(c for c in g["dt"] if (c["L"], c["N"], c["Tx"], c["phase_order"]) == (L, N, T, order))
    burn, blocks, block = 500, 200, 250
    times = [burn + k * block for k in range(blocks + 1)]
    vs, ws = [], []
    for seed in range(16):
        ts, s1, s2, w2 = _series(L, N, 128, 4242 + seed, times, T=T, order=order)
        v = (s1[-1].astype(float) - s1[0].astype(float)) / (L * L * (times[-1] - times[0]))
        vs.append(v.mean())
        ws.append(w2[1:].mean())
    vs, ws = np.array(vs), np.array(ws)
    dv, dw = vs.std(ddof=1) / 4, ws.std(ddof=1) / 4
    assert abs(vs.mean() - case["velocity"]) < 5 * dv + 1e-9, (vs.mean(), dv, case["velocity"])
    assert abs(ws.mean() - case["w2"]) < 5 * dw + 1e-9, (ws.mean(), dw, case["w2"])


def test_growth_exponent_near_paper():
    times = [64, 128, 256, 512, 1024, 2048]
    w = []
    for seed in range(2):
        ts, s1, s2, w2 = _series(4096, 1, 64, 100 + seed, times)
        w.append(w2.mean(axis=1))
    W2 = np.mean(w, axis=0)
    # Eq. 9 with t_{i/2}: local slopes of ln W against ln t
    beff = [0.5 * (math.log(W2[k]) - math.log(W2[k - 1])) / math.log(2.0) for k in range(1, len(times))]
    late = np.mean(beff[-3:])
    assert 0.20 < late < 0.27, beff


def test_roughness_exponent_near_paper():
    Ls = [32, 64, 128, 256]
    wsat = []
    for L in Ls:
        t_sat = int(20 * L ** 1.61)  # well past t_steady ~ L^z (z = alpha / beta ~ 1.6)
        times = [t_sat + k * max(1, t_sat // 40) for k in range(41)]
        ts, s1, s2, w2 = _series(L, 1, 64, 7 + L, times)
        wsat.append(math.sqrt(w2.mean()))
    slope = np.polyfit(np.log(Ls), np.log(wsat), 1)[0]
    assert 0.36 < slope < 0.42, (slope, wsat)
