"""Experiment drivers of section III on the library: growth runs (W^2 at the
paper's measurement times and the effective growth exponent), steady-state
widths and their finite-size scaling (the roughness exponent), and the
decomposition check (the same scaling on several tilings, section III.C).

Host orchestration only: every sweep and every exact measurement runs in the
library's kernels; this module chooses parameters and times and reduces the
exact sums the library returns with ``analysis``.  Surfaces of one job share
the selected sites (section II), so they are correlated samples; the paper
averages over them as realizations, and the errors here do the same.

    python -m paper_1605_02620_gb300.experiments growth --L 4096 --N 1 --t-max 10000
    python -m paper_1605_02620_gb300.experiments fss --Ls 32 64 128 256 --surfaces 1024
    python -m paper_1605_02620_gb300.experiments dd --Ls 64 128 --tilings 8x8 16x16 6x10+1
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import analysis
from . import rsos_free, rsos_init, rsos_params, rsos_read_series, rsos_schedule, rsos_sweep
from .inputs import paper_schedule


def _run(L, N, surfaces, times, seed, tile, tiling, stream=None):
    """One job from the flat start, measured at ``times`` (ascending); returns
    (times, w2[len(times)][surfaces]) from the exact sums."""
    times = [int(t) for t in times]
    p = rsos_params(L=L, N=N, surfaces=surfaces, tile=tile, seed=seed, series_capacity=len(times) + 1,
                    tiling=tiling)
    h = rsos_init(p, stream=stream)
    try:
        rsos_schedule(h, times)
        rsos_sweep(h, times[-1], stream=stream)
        ts, _, _, w2 = rsos_read_series(h, surfaces, len(times) + 1, stream=stream)
    finally:
        rsos_free(h)
    return [int(t) for t in ts], np.asarray(w2, dtype=np.float64)


def growth(L: int, N: int, t_max: int, surfaces: int = 64, seed: int = 0, tile=8, tiling: int = 0,
           m: float = 0.01, stream=None) -> dict:
    """Growth regime (Eq. 9): W^2 averaged over the surfaces at the paper's
    measurement times (Eq. 10 with exponent m) up to t_max, its standard
    error, and the effective exponent beta_eff from local slopes."""
    times = [t for t in paper_schedule(t_max, m=m) if t > 0]
    ts, w2 = _run(L, N, surfaces, times, seed, tile, tiling, stream)
    mean = w2.mean(axis=1)
    err = np.array([analysis.standard_error(row) for row in w2])
    t_mid, beff = analysis.beta_eff(ts, mean)
    return {"L": L, "N": N, "surfaces": surfaces, "tile": tile, "tiling": tiling, "t": ts,
            "w2": mean.tolist(), "w2_err": err.tolist(), "beta_eff_t": t_mid.tolist(),
            "beta_eff": beff.tolist()}


def steady_width(L: int, N: int, t_start: int, n_samples: int = 40, every: int = 0, surfaces: int = 64,
                 seed: int = 0, tile=8, tiling: int = 0, stream=None) -> dict:
    """Steady state (Eq. 12): W^2 sampled every ``every`` sweeps (default
    t_start / 40) from t_start on, averaged over samples and surfaces, with
    the per-surface time averages as the samples of its error."""
    every = every or max(1, t_start // 40)
    times = [t_start + k * every for k in range(n_samples)]
    ts, w2 = _run(L, N, surfaces, times, seed, tile, tiling, stream)
    per_surface = w2.mean(axis=0)
    return {"L": L, "N": N, "t": ts, "w2": float(w2.mean()), "w2_err": analysis.standard_error(per_surface),
            "w2_samples": w2.reshape(-1).tolist()}


def fss(Ls, N: int = 1, surfaces: int = 64, seed: int = 0, tile=8, tiling: int = 0, t_factor: float = 20.0,
        z: float = 1.61, n_samples: int = 40, stream=None) -> dict:
    """Finite-size scaling of the saturated width (Eq. 12): for every L a
    steady-state run started at t_factor * L^z sweeps (past t_steady ~ L^z,
    z = alpha / beta), then the local slopes alpha_eff between L and L/2, the
    least-squares slope of ln W against ln L, and the skewness and kurtosis
    of P(W^2) per L (section III.C)."""
    Ls = sorted(int(L) for L in Ls)
    rows = []
    for L in Ls:
        r = steady_width(L, N, int(math.ceil(t_factor * L ** z)), n_samples=n_samples, surfaces=surfaces,
                         seed=seed + L, tile=tile, tiling=tiling, stream=stream)
        S, Q = analysis.distribution_shape(r.pop("w2_samples"))
        r.update(S=S, Q=Q)
        rows.append(r)
    w2 = [r["w2"] for r in rows]
    L_mid, a_eff = analysis.alpha_eff(Ls, w2)
    slope = float(np.polyfit(np.log(Ls), 0.5 * np.log(w2), 1)[0]) if len(Ls) >= 2 else float("nan")
    return {"N": N, "surfaces": surfaces, "tile": tile, "tiling": tiling, "rows": rows,
            "alpha_eff_L": L_mid.tolist(), "alpha_eff": a_eff.tolist(), "alpha_fit": slope}


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
        res = growth(a.L, a.N, a.t_max, surfaces=a.surfaces, seed=a.seed, tile=tile, tiling=tiling)
    elif a.cmd == "fss":
        res = fss(a.Ls, a.N, surfaces=a.surfaces, seed=a.seed, tile=tile, tiling=tiling, t_factor=a.t_factor)
    else:
        res = dd_consistency(a.Ls, [parse_tiling(s) for s in a.tilings], N=a.N, surfaces=a.surfaces, seed=a.seed,
                             t_factor=a.t_factor)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
