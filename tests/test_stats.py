"""The test utilities' estimators on series with known answers: AR(1)
processes x_t = a x_{t-1} + e_t, whose integrated autocorrelation time is
(1 + a) / (2 (1 - a)), and the binned error of their mean."""
import numpy as np
import pytest

from tests.stats import binned_mean, binned_variance, tau_int


def _ar1(a, n, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - a * a)
    for t in range(1, n):
        x[t] = a * x[t - 1] + e[t]
    return x


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9])
def test_tau_int_of_ar1(a):
    exact = (1 + a) / (2 * (1 - a))
    est = [tau_int(_ar1(a, 200_000, s)) for s in range(4)]
    assert abs(np.mean(est) - exact) < 0.05 * exact + 0.02, (est, exact)


def test_binned_error_matches_tau_int():
    """The binned standard error equals sqrt(2 tau var / n) for a series with
    bins much longer than tau."""
    a, n = 0.8, 400_000
    x = _ar1(a, n, 7)
    _, err = binned_mean(x, 50)
    tau = (1 + a) / (2 * (1 - a))
    expect = np.sqrt(2 * tau * x.var() / n)
    assert 0.75 * expect < err < 1.3 * expect, (err, expect)


def test_binned_variance_of_ar1():
    """Stationary AR(1) with unit innovations has variance 1 / (1 - a^2); the
    jackknife error of the binned estimate covers the deviation, and over
    independent series its spread matches the quoted error."""
    a = 0.5
    exact = 1.0 / (1.0 - a * a)
    vals, errs = [], []
    for s in range(6):
        v, e = binned_variance(_ar1(a, 200_000, 100 + s))
        vals.append(v)
        errs.append(e)
        assert abs(v - exact) < 4 * e, (v, e, exact)
    spread = np.std(vals, ddof=1)
    assert 0.4 * np.mean(errs) < spread < 2.5 * np.mean(errs), (spread, errs)
