"""Analysis of measured width series and height power sums (section III).

Host-side arithmetic on the exact integers the library returns; nothing here
simulates.  Conventions follow the paper:

* effective exponents from local slopes of ln W (section II, the alpha_eff
  and beta_eff definitions): beta_eff between t and the latest measured time
  t' <= t / 2, alpha_eff between L and L / 2, each placed at the midpoint of
  its pair (the printed "(t_i - t_{i/2}) / 2" is read as the midpoint);
* the two-power-law correction form of Eq. 11,
  beta_eff(1/t) = beta + a1 / t^(4 beta) + a2 / t^beta;
* central moments Phi^n of a distribution and its skewness
  S = <Phi^3> / <Phi^2>^(3/2) and kurtosis Q = <Phi^4> / <Phi^2>^2 - 3
  (section III.C), for the height distribution (from exact power sums, the
  averages taken over surfaces and times) and for the width distribution
  P(W^2) (from per-surface W^2 samples);
* 1-sigma standard errors sqrt((<x^2> - <x>^2) / (n - 1)) over n independent
  samples (the printed formula reads as this).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .inputs import paper_schedule


def schedule(t_max: int, m: float = 0.01) -> list:
    """Measurement times of the paper (Eq. 10, section II): the same list as
    inputs.paper_schedule, t = 0 included."""
    return paper_schedule(t_max, m=m)


def jackknife(samples, estimator):
    """Delete-one jackknife over the first axis of ``samples`` (one entry per
    independent job): the estimate on the mean of all entries and its
    standard error sqrt((n - 1) / n * sum_k (e_k - e_mean)^2), e_k the
    estimate on the mean of all entries but k.  estimator maps a mean (one
    entry's shape) to a number or an array."""
    x = np.asarray(samples, dtype=np.float64)
    n = x.shape[0]
    if n < 2:
        raise ValueError("the jackknife needs at least two samples")
    full = np.asarray(estimator(x.mean(axis=0)), dtype=np.float64)
    total = x.sum(axis=0)
    reps = np.array([np.asarray(estimator((total - x[k]) / (n - 1)), dtype=np.float64) for k in range(n)])
    err = np.sqrt((n - 1) / n * ((reps - reps.mean(axis=0)) ** 2).sum(axis=0))
    if full.ndim == 0:
        return float(full), float(err)
    return full, err


def standard_error(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 2:
        return float("nan")
    return float(np.sqrt(max(0.0, x.var()) / (n - 1)))


def beta_eff(times, w2):
    """Local slopes of ln W against ln t (W^2 series of one surface or an
    average).  Returns (t_mid, beta_eff) for every time t > 0 that has an
    earlier measured time t' <= t / 2 (t' > 0): the slope between t' and the
    latest such t'."""
    t = np.asarray(times, dtype=np.float64)
    w = np.sqrt(np.asarray(w2, dtype=np.float64))
    mids, slopes = [], []
    for i in range(len(t)):
        if t[i] <= 0:
            continue
        j = np.searchsorted(t, t[i] / 2.0, side="right") - 1
        if j < 0 or t[j] <= 0 or t[j] >= t[i] or w[j] <= 0 or w[i] <= 0:
            continue
        mids.append(0.5 * (t[i] + t[j]))
        slopes.append((np.log(w[i]) - np.log(w[j])) / (np.log(t[i]) - np.log(t[j])))
    return np.array(mids), np.array(slopes)


def alpha_eff(Ls, w2_sat):
    """Local slopes of the saturated ln W against ln L for every L whose half
    L / 2 is also given.  Returns (L_mid, alpha_eff)."""
    pairs = dict(zip((int(v) for v in Ls), (float(v) for v in w2_sat)))
    mids, slopes = [], []
    for L in sorted(pairs):
        if L % 2 == 0 and L // 2 in pairs:
            mids.append(0.5 * (L + L / 2))
            slopes.append(0.5 * (np.log(pairs[L]) - np.log(pairs[L // 2])) / np.log(2.0))
    return np.array(mids), np.array(slopes)


def fit_beta_two_power_laws(t_mid, beff, beta_grid=None):
    """Least-squares fit of Eq. 11, beta_eff = beta + a1 t^(-4 beta) + a2 t^(-beta):
    for a fixed beta the amplitudes follow from a linear least-squares problem,
    so beta is scanned on a grid and refined by a golden-section search on the
    residual.  Returns (beta, a1, a2, rms residual)."""
    t = np.asarray(t_mid, dtype=np.float64)
    y = np.asarray(beff, dtype=np.float64)

    def solve(b):
        # the constant term is the exponent itself: fit y - b = a1 x1 + a2 x2
        A = np.stack([t ** (-4.0 * b), t ** (-b)], axis=1)
        c, *_ = np.linalg.lstsq(A, y - b, rcond=None)
        r = y - b - A @ c
        return float(np.sqrt(np.mean(r * r))), c

    grid = np.linspace(0.15, 0.35, 201) if beta_grid is None else np.asarray(beta_grid, dtype=np.float64)
    errs = [solve(b)[0] for b in grid]
    k = int(np.argmin(errs))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(80):
        if solve(c)[0] < solve(d)[0]:
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    best = 0.5 * (a + b)
    rms, (a1, a2) = solve(best)
    return best, float(a1), float(a2), rms


def central_moments(power_sums, L: int):
    """Exact central moments (Phi^2, Phi^3, Phi^4) of one surface's height
    distribution over its L^2 sites, from [sum h, sum h^2, sum h^3, sum h^4]."""
    n = int(L) * int(L)
    s1, s2, s3, s4 = (int(v) for v in power_sums)
    m1 = Fraction(s1, n)
    m2, m3, m4 = Fraction(s2, n), Fraction(s3, n), Fraction(s4, n)
    p2 = m2 - m1 ** 2
    p3 = m3 - 3 * m1 * m2 + 2 * m1 ** 3
    p4 = m4 - 4 * m1 * m3 + 6 * m1 ** 2 * m2 - 3 * m1 ** 4
    return p2, p3, p4


def height_shape(power_sum_rows, L: int):
    """Skewness S_h and kurtosis Q_h of the height distribution (section
    III.C): <Phi^3> / <Phi^2>^(3/2) and <Phi^4> / <Phi^2>^2 - 3, the averages
    over every (surface, time) given.  power_sum_rows: iterable of
    [sum h, sum h^2, sum h^3, sum h^4].  Returns (S_h, Q_h, <Phi^2>)."""
    acc = [Fraction(0), Fraction(0), Fraction(0)]
    n = 0
    for ps in power_sum_rows:
        for k, v in enumerate(central_moments(ps, L)):
            acc[k] += v
        n += 1
    p2, p3, p4 = (float(a / n) for a in acc)
    return p3 / p2 ** 1.5, p4 / p2 ** 2 - 3.0, p2


def distribution_shape(samples):
    """Skewness S and kurtosis Q of the distribution of the given samples
    (for P(W^2): per-surface W^2 values), Phi^n about the sample mean."""
    x = np.asarray(samples, dtype=np.float64)
    d = x - x.mean()
    p2, p3, p4 = (float(np.mean(d ** k)) for k in (2, 3, 4))
    return p3 / p2 ** 1.5, p4 / p2 ** 2 - 3.0
