"""Pins of the oracle's error analysis (blocking and the ratio estimator).

The paper gives no error analysis for E_proj (Eq. (9)); the oracle's reading
is Flyvbjerg-Petersen blocking with the optimal-block rule of Lee et al.
(2011) and a delta-method error for the ratio of means with the covariance of
the two means taken at one blocking level.  These tests pin it to what the
mathematics fixes, not to a retyped formula:

* independent normal samples: sigma = s / sqrt(n);
* a stationary AR(1) series x_t = rho x_{t-1} + e_t: the variance of its mean
  is known in closed form, sigma_x^2 / n [(1 + rho)/(1 - rho)
  - 2 rho (1 - rho^n) / (n (1 - rho)^2)], sigma_x^2 = 1 / (1 - rho^2);
* coverage: over an ensemble of independent series, |mean - mu| < 2 sigma
  must hold for about 95.4 % of them (a plateau picked too early, or a sigma
  too small, lowers it; a sigma too large raises it);
* the ratio estimator against the spread of the ratio over an ensemble, for
  strongly correlated numerator and denominator (the case of E_proj), where
  an error that leaves out or mis-signs the covariance is off by a factor of
  several.

Planted mistakes (sigma x 2 or / 2, level 0 as the plateau, the covariance
term dropped) are checked to fail the same criteria.
"""
import math

import numpy as np
import pytest
from scipy.signal import lfilter

import oracle


def ar1(rng, reps, n, rho, scale=1.0):
    """reps independent stationary AR(1) series of length n (unit innovations x scale)."""
    e = rng.normal(0.0, scale, size=(reps, n))
    x0 = e[:, 0] / math.sqrt(1.0 - rho * rho)
    x = lfilter([1.0], [1.0, -rho], e[:, 1:], axis=1, zi=(rho * x0)[:, None])[0]
    return np.concatenate([x0[:, None], x], axis=1)


def ar1_sigma_of_mean(n, rho, scale=1.0):
    s2 = scale * scale / (1.0 - rho * rho)
    return math.sqrt(s2 / n * ((1.0 + rho) / (1.0 - rho) - 2.0 * rho * (1.0 - rho ** n) / (n * (1.0 - rho) ** 2)))


def sigmas(series, f=None):
    f = f or (lambda x: oracle.blocking(x)[1])
    return np.array([f(x) for x in series])


def test_levels_halve_and_drop_the_odd_element():
    x = np.arange(11, dtype=np.float64)
    lev = oracle.blocking_levels(x)
    assert [y.size for y in lev] == [11, 5, 2]
    np.testing.assert_array_equal(lev[1], [0.5, 2.5, 4.5, 6.5, 8.5])
    np.testing.assert_array_equal(lev[2], [1.5, 5.5])


def test_constant_and_short_series():
    m, s, _ = oracle.blocking(np.full(64, 3.25))
    assert m == 3.25 and s == 0.0
    m, s, errs = oracle.blocking([1.0, 3.0])
    assert m == 2.0 and s == 1.0 and errs == [1.0]   # sqrt(var_pop / (n - 1)) = sqrt(1 / 1)


@pytest.mark.parametrize("n", [1024, 8192])
def test_independent_samples(n):
    rng = np.random.default_rng(100 + n)
    x = rng.normal(0.0, 2.0, size=(400, n))
    s = sigmas(x)
    true = 2.0 / math.sqrt(n)
    assert abs(np.mean(s) / true - 1.0) < 0.03, np.mean(s) / true
    assert abs(np.mean(2.0 * s) / true - 1.0) > 0.5 and abs(np.mean(0.5 * s) / true - 1.0) > 0.3


@pytest.mark.parametrize("rho,n", [(0.9, 4096), (0.9, 16384), (0.98, 16384)])
def test_ar1_sigma_of_the_mean(rho, n):
    rng = np.random.default_rng(int(rho * 1000) + n)
    x = ar1(rng, 400, n, rho)
    s = sigmas(x)
    true = ar1_sigma_of_mean(n, rho)
    assert 0.92 < np.mean(s) / true < 1.04, (np.mean(s) / true)
    # the ensemble's own spread of the means agrees with the closed form
    assert abs(np.std(np.mean(x, axis=1)) / true - 1.0) < 0.1
    # level 0 (no blocking) underestimates by sqrt(tau_int)
    s0 = sigmas(x, lambda y: oracle.blocking(y)[2][0])
    assert np.mean(s0) / true < 0.5


def test_ar1_coverage():
    rng = np.random.default_rng(77)
    n, rho, reps = 8192, 0.95, 2000
    x = ar1(rng, reps, n, rho)
    m = np.mean(x, axis=1)
    s = sigmas(x)
    cover = float(np.mean(np.abs(m) < 2.0 * s))
    # 95.4 % for a known sigma; the estimate from ~16 blocks (a t distribution
    # with ~15 degrees of freedom) gives about 93.6 %
    assert 0.92 < cover < 0.975, cover
    # planted: a plateau at block length 8 (below tau_int ~ 39), and sigma halved
    early = sigmas(x, lambda y: oracle.blocking(y)[2][3])
    assert float(np.mean(np.abs(m) < 2.0 * early)) < 0.8
    assert float(np.mean(np.abs(m) < 1.0 * s)) < 0.8


def ratio_ensemble(rng, reps, n):
    """den = 10 + a, num = -20 - 2 a + b with a, b independent AR(1) (rho 0.9):
    num/den fluctuates only through b, so sigma(r) = sigma(mean b) / 10."""
    a = ar1(rng, reps, n, 0.9)
    b = ar1(rng, reps, n, 0.9, scale=0.3)
    return -20.0 - 2.0 * a + b, 10.0 + a


def test_ratio_estimator_against_the_ensemble():
    rng = np.random.default_rng(9)
    reps, n = 600, 8192
    num, den = ratio_ensemble(rng, reps, n)
    est = [oracle.ratio_estimate(num[i], den[i]) for i in range(reps)]
    r = np.array([e[0] for e in est])
    s = np.array([e[1] for e in est])
    spread = float(np.std(r))
    assert abs(np.mean(s) / spread - 1.0) < 0.1, (np.mean(s), spread)
    # ratio of expectations: -2; coverage of it
    cover = float(np.mean(np.abs(r + 2.0) < 2.0 * s))
    assert 0.92 < cover < 0.985, cover
    # planted: the covariance of the two means left out
    def no_cov(x, y):
        mn, md = np.mean(x), np.mean(y)
        _, sn, _ = oracle.blocking(x)
        _, sd, _ = oracle.blocking(y)
        rr = mn / md
        return math.sqrt(sn * sn + rr * rr * sd * sd) / abs(md)
    s_bad = np.array([no_cov(num[i], den[i]) for i in range(50)])
    assert np.mean(s_bad) / spread > 3.0
