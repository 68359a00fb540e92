"""Experiment drivers of section III on the library: growth runs (W^2 at the
paper's measurement times and the growth exponent), steady-state widths and
their finite-size scaling (the roughness exponent), and the decomposition
check (the same scaling on several tilings, section III.C).

Host orchestration only: every sweep and every exact measurement runs in the
library's kernels; this module chooses parameters and times and reduces the
exact sums the library returns with ``analysis``.

Errors.  The surfaces of one job share the selected sites (section II), so
they are correlated samples of one Markov chain.  Every estimate here is
therefore made from several independent jobs (different seeds; advanced
together as one batch): each job contributes one sample (its mean over its
surfaces), standard errors are the spread over jobs, and the errors of the
exponents (local slopes and fits) are delete-one-job jackknife errors.

    python -m paper_1605_02620_gb300.experiments growth --L 4096 --N 1 --t-max 10000 --jobs 8
    python -m paper_1605_02620_gb300.experiments fss --Ls 32 64 128 256 512 --surfaces 64 --jobs 16
    python -m paper_1605_02620_gb300.experiments dd --Ls 64 128 --tilings 8x8 16x16 6x10+1
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import analysis
from . import (rsos_batch_create, rsos_batch_free, rsos_batch_job, rsos_batch_poll, rsos_batch_run,
               rsos_batch_schedule, rsos_params, rsos_read_series)
from .inputs import paper_schedule


def _run_jobs(L, N, surfaces, times, seeds, tile, tiling, stream=None):
    """Independent jobs (one per seed) from the flat start, measured at
    ``times`` (ascending), advanced together as one batch.  Returns
    (times, w2[jobs][len(times)][surfaces]) from the exact sums."""
    times = [int(t) for t in times]
    params = [rsos_params(L=L, N=N, surfaces=surfaces, tile=tile, seed=s, series_capacity=len(times) + 1,
                          tiling=tiling) for s in seeds]
    b = rsos_batch_create(params, [times[-1]] * len(params))
    try:
        for k in range(len(params)):
            rsos_batch_schedule(b, k, times)
        rsos_batch_run(b, stream)
        done = set()
        while len(done) < len(params):
            _, ids = rsos_batch_poll(b)
            done |= set(ids)
            if len(done) < len(params):
                time.sleep(0.002)
        w2 = []
        for k in range(len(params)):
            ts, _, _, w = rsos_read_series(rsos_batch_job(b, k), surfaces, len(times) + 1, stream)
            if [int(t) for t in ts] != times:
                raise RuntimeError(f"job {k} measured at {list(ts)}, expected {times}")
            w2.append(np.asarray(w, dtype=np.float64))
    finally:
        rsos_batch_free(b)
    return times, np.stack(w2)


def _slope(x, y):
    """Least-squares slope of y against x."""
    return float(np.polyfit(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64), 1)[0])


def growth(L: int, N: int, t_max: int, surfaces: int = 64, jobs: int = 8, seed: int = 0, tile=8, tiling: int = 0,
           m: float = 0.01, window=None, stream=None) -> dict:
    """Growth regime (Eq. 9): W^2 at the paper's measurement times (Eq. 10
    with exponent m) up to t_max, averaged over the surfaces of `jobs`
    independent jobs, with its standard error over jobs; the effective
    exponent beta_eff from local slopes, with jackknife errors; and the growth
    exponent fitted over a window of times: the slope of ln W against ln t
    (beta_fit) and the two-correction form of Eq. 11 (beta_eq11), each with
    its jackknife error.  window = (t_lo, t_hi), default the last decade."""
    times = [t for t in paper_schedule(t_max, m=m) if t > 0]
    if len(times) < 2:
        raise ValueError(f"t_max = {t_max} leaves fewer than two measurement times of Eq. 10 (m = {m})")
    if jobs < 2:
        raise ValueError("the errors need at least two independent jobs")
    ts, w2 = _run_jobs(L, N, surfaces, times, [seed + k for k in range(jobs)], tile, tiling, stream)
    per_job = w2.mean(axis=2)  # [jobs][times]
    mean = per_job.mean(axis=0)
    err = per_job.std(axis=0, ddof=1) / math.sqrt(jobs)
    t_mid, beff = analysis.beta_eff(ts, mean)
    beff_err = analysis.jackknife(per_job, lambda c: analysis.beta_eff(ts, c)[1])[1]
    t_lo, t_hi = window if window else (t_max / 10.0, t_max)
    sel = [i for i, t in enumerate(ts) if t_lo <= t <= t_hi]
    if len(sel) < 3:
        raise ValueError(f"the fit window {t_lo}..{t_hi} holds fewer than three measurement times")
    lt = np.log(np.asarray(ts, dtype=np.float64)[sel])
    fit = lambda c: 0.5 * _slope(lt, np.log(np.asarray(c)[sel]))  # noqa: E731
    beta_fit, beta_fit_err = analysis.jackknife(per_job, fit)
    # Eq. 11 on the local slopes from t >= 10 (the fit's own lower cut)
    late = lambda c: [(tm, b) for tm, b in zip(*analysis.beta_eff(ts, c)) if tm >= 10.0]  # noqa: E731
    eq11 = lambda c: analysis.fit_beta_two_power_laws(*zip(*late(c)))[0]  # noqa: E731
    beta_eq11, beta_eq11_err = analysis.jackknife(per_job, eq11)
    return {"L": L, "N": N, "surfaces": surfaces, "jobs": jobs, "tile": tile, "tiling": tiling, "t": ts,
            "w2": mean.tolist(), "w2_err": err.tolist(), "beta_eff_t": t_mid.tolist(), "beta_eff": beff.tolist(),
            "beta_eff_err": np.asarray(beff_err).tolist(), "window": [t_lo, t_hi], "beta_fit": beta_fit,
            "beta_fit_err": beta_fit_err, "beta_eq11": beta_eq11, "beta_eq11_err": beta_eq11_err}


def steady_width(L: int, N: int, t_start: int, n_samples: int = 40, every: int = 0, surfaces: int = 64,
                 jobs: int = 8, seed: int = 0, tile=8, tiling: int = 0, stream=None) -> dict:
    """Steady state (Eq. 12): W^2 sampled every ``every`` sweeps (default
    t_start / 40) from t_start on, in `jobs` independent jobs.  Each job's
    time and surface average is one sample: w2 is their mean, w2_err their
    standard error; w2_jobs lists them."""
    every = every or max(1, t_start // 40)
    times = [t_start + k * every for k in range(n_samples)]
    ts, w2 = _run_jobs(L, N, surfaces, times, [seed + k for k in range(jobs)], tile, tiling, stream)
    per_job = w2.mean(axis=(1, 2))
    return {"L": L, "N": N, "t": ts, "jobs": jobs, "w2": float(per_job.mean()),
            "w2_err": analysis.standard_error(per_job), "w2_jobs": per_job.tolist(),
            "w2_samples": w2.reshape(-1).tolist()}


def fss(Ls, N: int = 1, surfaces: int = 64, jobs: int = 8, seed: int = 0, tile=8, tiling: int = 0,
        t_factor: float = 20.0, z: float = 1.61, n_samples: int = 40, stream=None) -> dict:
    """Finite-size scaling of the saturated width (Eq. 12): for every L,
    `jobs` independent steady-state runs started at t_factor * L^z sweeps
    (past t_steady ~ L^z, z = alpha / beta); then the local slopes alpha_eff
    between L and L/2 and the least-squares slope alpha_fit of ln W against
    ln L, each with its jackknife error over jobs, and the skewness and
    kurtosis of P(W^2) per L (section III.C)."""
    Ls = sorted(int(L) for L in Ls)
    if jobs < 2:
        raise ValueError("the errors need at least two independent jobs")
    rows = []
    for L in Ls:
        r = steady_width(L, N, int(math.ceil(t_factor * L ** z)), n_samples=n_samples, surfaces=surfaces,
                         jobs=jobs, seed=seed + 1000 * L, tile=tile, tiling=tiling, stream=stream)
        S, Q = analysis.distribution_shape(r.pop("w2_samples"))
        r.update(S=S, Q=Q)
        rows.append(r)
    per_job = np.array([r["w2_jobs"] for r in rows]).T  # [jobs][Ls]: job k of every L is one jackknife unit
    w2 = per_job.mean(axis=0)
    L_mid, a_eff = analysis.alpha_eff(Ls, w2)
    a_err = analysis.jackknife(per_job, lambda c: analysis.alpha_eff(Ls, c)[1])[1]
    lL = np.log(np.asarray(Ls, dtype=np.float64))
    if len(Ls) >= 2:
        alpha_fit, alpha_err = analysis.jackknife(per_job, lambda c: 0.5 * _slope(lL, np.log(c)))
    else:
        alpha_fit, alpha_err = float("nan"), float("nan")
    return {"N": N, "surfaces": surfaces, "jobs": jobs, "tile": tile, "tiling": tiling, "rows": rows,
            "alpha_eff_L": L_mid.tolist(), "alpha_eff": a_eff.tolist(), "alpha_eff_err": np.asarray(a_err).tolist(),
            "alpha_fit": alpha_fit, "alpha_fit_err": alpha_err}


def dd_consistency(Ls, tilings, **kw) -> dict:
    """The decomposition check of section III.C: the same finite-size scaling
    on several tilings, each a (tile, tiling) pair such as (8, 0), (16, 0) or
    ((6, 10), 1) for 6(+1) x 10(+1)."""
    out = []
    for tile, tiling in tilings:
        out.append(fss(Ls, tile=tile, tiling=tiling, **kw))
    return {"tilings": out}


def parse_tiling(spec: str):
    """'8' or '8x8' -> (8, 0); '6x10+1' -> ((6, 10), 1) (a (+1) tiling)."""
    plus = spec.endswith("+1")
    body = spec[:-2] if plus else spec
    parts = [int(v) for v in body.lower().split("x")]
    if len(parts) == 1:
        parts = parts * 2
    if len(parts) != 2:
        raise ValueError(f"bad tiling {spec!r}")
    tile = parts[0] if (parts[0] == parts[1] and not plus) else tuple(parts)
    return tile, 1 if plus else 0


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1605_02620_gb300.experiments")
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("growth")
    g.add_argument("--L", type=int, default=4096)
    g.add_argument("--t-max", type=int, default=10000)
    for sp in (g, sub.add_parser("fss"), sub.add_parser("dd")):
        sp.add_argument("--N", type=int, default=1)
        sp.add_argument("--surfaces", type=int, default=64)
        sp.add_argument("--jobs", type=int, default=8)
        sp.add_argument("--seed", type=int, default=0)
        if sp is not g:
            sp.add_argument("--Ls", type=int, nargs="+", default=[32, 64, 128, 256])
            sp.add_argument("--t-factor", type=float, default=20.0)
        sp.add_argument("--tiling", default="8x8", help="8x8, 16x16, 6x10+1 ... (dd: --tilings)")
        if sp.prog.endswith("dd"):
            sp.add_argument("--tilings", nargs="+", default=["8x8", "16x16", "6x10+1"])
    a = ap.parse_args(argv)
    tile, tiling = parse_tiling(a.tiling)
    if a.cmd == "growth":
        res = growth(a.L, a.N, a.t_max, surfaces=a.surfaces, jobs=a.jobs, seed=a.seed, tile=tile, tiling=tiling)
    elif a.cmd == "fss":
        res = fss(a.Ls, a.N, surfaces=a.surfaces, jobs=a.jobs, seed=a.seed, tile=tile, tiling=tiling,
                  t_factor=a.t_factor)
    else:
        res = dd_consistency(a.Ls, [parse_tiling(s) for s in a.tilings], N=a.N, surfaces=a.surfaces, jobs=a.jobs,
                             seed=a.seed, t_factor=a.t_factor)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
