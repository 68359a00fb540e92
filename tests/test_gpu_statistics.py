"""Statistical checks of the CUDA path against exact results and against the
paper's exponents (section III).  Seeds are fixed, so the outcomes are
deterministic.

* Tiny lattices: the GPU's DT dynamics reproduces the exact stationary growth
  velocity and squared width of the enumerated Markov chains.
* Growth regime (Eq. 9): the growth exponent fitted to W(t) over the last
  decade of a run at L = 4096 (N = 1, t = 1e3..1e4, eight independent jobs,
  jackknife error over jobs) agrees with the paper's beta_1 = 0.2415(5)
  (Table I) within three combined standard errors.
* Steady state (Eq. 12): the roughness exponent fitted to the saturated
  width over L = 32..256 (eight independent jobs per L, jackknife error)
  agrees with the paper's direct N = 1 fit alpha = 0.392(1) (section III.B)
  within three combined standard errors.
* Decomposition check (section III.C): the same steady-state scaling on
  8 x 8, 16 x 16 and 6(+1) x 10(+1) tiles (L = 64 and 128, the paper's
  smallest sizes for this check, 512 realizations per L) gives roughness
  exponents that agree with the paper's alpha = 0.390(4) and with each
  other; the saturated width is larger on 16 x 16 tiles, whose larger
  sub-tiles bring the double-tiling amplitude closer to random-sequential
  updating.
Each test prints the fit, its error and the paper's value.
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


def _within(fit, err, paper, paper_err, what, k=3.0):
    sigma = math.hypot(err, paper_err)
    print(f"{what}: fit {fit:.4f} +- {err:.4f}, paper {paper} +- {paper_err}, distance {abs(fit - paper) / sigma:.2f} sigma")
    assert err > 0 and abs(fit - paper) < k * sigma, (what, fit, err, paper, paper_err)


def test_growth_exponent_fit_agrees_with_paper():
    from paper_1605_02620_gb300 import experiments as E
    r = E.growth(4096, 1, 10000, surfaces=64, jobs=8, seed=100, window=(1000, 10000))
    _within(r["beta_fit"], r["beta_fit_err"], 0.2415, 0.0005, "beta (N = 1, L = 4096, t = 1e3..1e4)")


def test_roughness_exponent_fit_agrees_with_paper():
    from paper_1605_02620_gb300 import experiments as E
    r = E.fss([32, 64, 128, 256], N=1, surfaces=64, jobs=8, seed=7)
    _within(r["alpha_fit"], r["alpha_fit_err"], 0.392, 0.001, "alpha (N = 1, L = 32..256)")
    # the local slopes between L and L/2 are each consistent with the fit
    for a, e in zip(r["alpha_eff"], r["alpha_eff_err"]):
        assert abs(a - r["alpha_fit"]) < 4 * e, (r["alpha_eff"], r["alpha_eff_err"])


@pytest.mark.slow
def test_decomposition_check_agrees_across_tilings():
    from paper_1605_02620_gb300 import experiments as E
    tilings = [(8, 0), (16, 0), ((6, 10), 1)]
    r = E.dd_consistency([64, 128], tilings, N=1, surfaces=64, jobs=8, seed=11)["tilings"]
    names = ["8 x 8", "16 x 16", "6(+1) x 10(+1)"]
    for name, f in zip(names, r):
        _within(f["alpha_fit"], f["alpha_fit_err"], 0.390, 0.004, f"alpha on {name} tiles (L = 64, 128)")
    base = r[0]
    for name, f in zip(names[1:], r[1:]):
        sigma = math.hypot(f["alpha_fit_err"], base["alpha_fit_err"])
        print(f"{name} against 8 x 8: {abs(f['alpha_fit'] - base['alpha_fit']) / sigma:.2f} sigma")
        assert abs(f["alpha_fit"] - base["alpha_fit"]) < 3 * sigma, (name, f["alpha_fit"], base["alpha_fit"])
    # the amplitude depends on the sub-tile (1 - 1/(2a) for a-site sub-tiles
    # as N grows without bound): wider on 16 x 16 than on 8 x 8 at every L
    for a8, a16 in zip(base["rows"], r[1]["rows"]):
        assert a16["w2"] - a8["w2"] > 3 * math.hypot(a16["w2_err"], a8["w2_err"]), (a8["L"], a8["w2"], a16["w2"])
