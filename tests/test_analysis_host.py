"""The analysis layer (local slopes, Eq. 11, distribution shapes) on inputs
whose answers are fixed by closed forms or by library routines."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1605_02620_gb300 import analysis as A


def test_schedule_follows_the_recursion():
    ts = A.schedule(100000)
    assert ts[0] == 0 and ts[-1] <= 100000 and all(b > a for a, b in zip(ts, ts[1:]))
    # t_{i+1} = (t_i + 10) e^0.01: the first real times are 0, 10.1005, 20.30, ...
    assert ts[1:4] == [11, 21, 31]
    # dt/di ~ 0.01 t + 10: about 100 ln((0.01 * 1e5 + 10) / (0.01 * 1e3 + 10)) = 392 points in [1e3, 1e5]
    n = sum(1 for t in ts if 1000 <= t <= 100000)
    assert abs(n - 100 * math.log(1010 / 20)) < 3


def test_schedule_is_the_inputs_schedule():
    from paper_1605_02620_gb300.inputs import paper_schedule
    for t_max in (0, 5, 11, 1000, 123457):
        for m in (0.01, 0.05):
            assert A.schedule(t_max, m=m) == paper_schedule(t_max, m=m)


def test_jackknife_of_the_mean_is_the_standard_error():
    # for the mean (a linear estimator) the delete-one jackknife error equals
    # the standard error s / sqrt(n) exactly, entry by entry
    rng = np.random.Generator(np.random.PCG64(11))
    x = rng.normal(3.0, 2.0, size=(9, 5))
    est, err = A.jackknife(x, lambda c: c)
    assert np.allclose(est, x.mean(axis=0))
    assert np.allclose(err, x.std(axis=0, ddof=1) / math.sqrt(9), rtol=1e-12)
    # a scalar linear functional: the same identity
    w = np.array([1.0, -2.0, 0.5, 3.0, 1.0])
    e, s = A.jackknife(x, lambda c: float(w @ c))
    assert e == pytest.approx(float(w @ x.mean(axis=0))) and s == pytest.approx((x @ w).std(ddof=1) / 3.0)
    with pytest.raises(ValueError):
        A.jackknife(x[:1], lambda c: c)


def test_jackknife_of_a_log_slope_matches_the_delta_method():
    # slope of ln y against ln x from noisy power laws: the jackknife error of
    # the slope agrees with the propagated error of independent samples
    rng = np.random.Generator(np.random.PCG64(12))
    xs = np.array([32.0, 64.0, 128.0, 256.0])
    n, rel = 400, 0.01
    samples = 0.9 * xs ** 0.78 * (1 + rel * rng.standard_normal((n, len(xs))))
    slope = lambda c: float(np.polyfit(np.log(xs), np.log(c), 1)[0])  # noqa: E731
    est, err = A.jackknife(samples, slope)
    lx = np.log(xs) - np.log(xs).mean()
    delta = rel / math.sqrt(n) * math.sqrt(float((lx ** 2).sum())) / float((lx ** 2).sum())
    assert est == pytest.approx(0.78, abs=5 * delta) and err == pytest.approx(delta, rel=0.15)


def test_beta_eff_of_a_power_law_is_exact():
    t = np.array(A.schedule(20000)[1:], dtype=float)
    for beta in (0.2415, 0.25, 1 / 3):
        mid, b = A.beta_eff(t, 3.7 * t ** (2 * beta))
        assert len(b) > 100 and np.allclose(b, beta, atol=1e-12)


def test_beta_eff_approaches_beta_with_corrections():
    # W = t^beta (1 + c t^-x): the local slope tends to beta like t^-x
    t = np.array(A.schedule(10 ** 6)[1:], dtype=float)
    beta, c, x = 0.24, 0.8, 0.25
    w2 = (t ** beta * (1 + c * t ** -x)) ** 2
    mid, b = A.beta_eff(t, w2)
    late = mid > 1e5
    assert np.all(np.abs(b[late] - beta) < 2 * c * x * mid[late] ** -x)
    assert abs(b[-1] - beta) < abs(b[len(b) // 4] - beta)


def test_alpha_eff_of_a_power_law():
    Ls = [32, 64, 128, 256, 512]
    mid, a = A.alpha_eff(Ls, [0.9 * L ** (2 * 0.39) for L in Ls])
    assert list(mid) == [48, 96, 192, 384] and np.allclose(a, 0.39, atol=1e-12)


def test_eq11_fit_recovers_its_parameters():
    t = np.geomspace(150, 1e5, 300)
    beta, a1, a2 = 0.2415, -0.9, 0.35
    y = beta + a1 * t ** (-4 * beta) + a2 * t ** (-beta)
    b, f1, f2, rms = A.fit_beta_two_power_laws(t, y)
    assert abs(b - beta) < 1e-6 and abs(f1 - a1) < 1e-3 and abs(f2 - a2) < 1e-4 and rms < 1e-8


def test_central_moments_closed_forms():
    L = 4
    # two-point field +-a: Phi2 = a^2, Phi3 = 0, Phi4 = a^4 (kurtosis -2)
    a = 7
    h = np.array([[a, -a] * 2] * 4, dtype=np.int64)[None]
    ps = O.power_sums(np.ascontiguousarray(h))[0]
    p2, p3, p4 = A.central_moments(ps, L)
    assert (p2, p3, p4) == (a * a, 0, a ** 4)
    # uniform on 0..15 (one site each): Phi2 = (n^2-1)/12, Phi4 = (n^2-1)(3n^2-7)/240
    n = 16
    h = np.arange(n, dtype=np.int64).reshape(1, 4, 4) + 10 ** 9  # a large offset must not matter
    p2, p3, p4 = A.central_moments(O.power_sums(h)[0], L)
    assert p2 == Fraction(n * n - 1, 12) and p3 == 0 and p4 == Fraction((n * n - 1) * (3 * n * n - 7), 240)


def test_height_shape_matches_scipy_on_oracle_surfaces():
    p = O.Params(L=32, N=1, Tx=8, Ty=8, seed=3)
    h = O.flat(32, 8)
    O.sweeps(p, h, list(range(8)), 0, 60)
    rows = O.power_sums(h)
    for j in range(8):
        S, Q, p2 = A.height_shape([rows[j]], 32)
        x = h[j].ravel().astype(float)
        assert math.isclose(S, stats.skew(x), rel_tol=1e-9, abs_tol=1e-12)
        assert math.isclose(Q, stats.kurtosis(x), rel_tol=1e-9, abs_tol=1e-12)
        assert math.isclose(p2, x.var(), rel_tol=1e-12)
    # central moments do not see a common shift of all heights
    shifted = O.power_sums(np.ascontiguousarray(h + 123456))
    for a, b in zip(rows, shifted):
        assert A.central_moments(a, 32) == A.central_moments(b, 32)


def test_distribution_shape_matches_scipy():
    rng = np.random.Generator(np.random.PCG64(7))
    x = rng.gamma(2.0, 1.5, size=5000)
    S, Q = A.distribution_shape(x)
    assert math.isclose(S, stats.skew(x), rel_tol=1e-10)
    assert math.isclose(Q, stats.kurtosis(x), rel_tol=1e-10)


def test_standard_error():
    x = np.array([1.0, 2.0, 3.0, 4.0])
    assert A.standard_error(x) == pytest.approx(math.sqrt(np.var(x) / 3))
