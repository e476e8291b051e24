"""Binning (blocking) estimates of the mean and its standard error for
correlated Monte Carlo series, and the integrated autocorrelation time
(the quantity behind the paper's tau_int trade-off, Sec. 3.4)."""
import numpy as np


def binned_mean(x, n_bins=50):
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // n_bins) * n_bins
    bins = x[:n].reshape(n_bins, -1).mean(axis=1)
    return float(bins.mean()), float(bins.std(ddof=1) / np.sqrt(n_bins))


def tau_int(x, c=6.0):
    """Integrated autocorrelation time tau = 1/2 + sum_{t >= 1} rho(t), the
    sum cut at the first window W >= c tau(W) (Sokal's automatic windowing).
    The variance of the mean of n samples is then 2 tau var(x) / n."""
    x = np.asarray(x, dtype=np.float64)
    x = x - x.mean()
    n = x.size
    f = np.fft.rfft(x, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    rho = acf / acf[0]
    tau = 0.5
    for w in range(1, n):
        tau += rho[w]
        if w >= c * tau:
            break
    return float(tau)


def assert_within(estimate, error, exact, nsigma=4.0, floor=0.0, what=""):
    dev = abs(estimate - exact)
    assert dev <= nsigma * error + floor, (
        f"{what}: {estimate} +- {error} vs exact {exact} ({dev / max(error, 1e-300):.2f} sigma)")


def binned_variance(x, n_bins=50):
    """Variance <x^2> - <x>^2 of a correlated series and its jackknife error
    over n_bins consecutive bins (each leave-one-bin-out estimate uses the
    means of x and x^2 over the other bins)."""
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // n_bins) * n_bins
    b1 = x[:n].reshape(n_bins, -1).mean(axis=1)
    b2 = (x[:n] ** 2).reshape(n_bins, -1).mean(axis=1)
    s1, s2 = b1.sum(), b2.sum()
    loo1 = (s1 - b1) / (n_bins - 1)
    loo2 = (s2 - b2) / (n_bins - 1)
    jk = loo2 - loo1 ** 2
    full = s2 / n_bins - (s1 / n_bins) ** 2
    err = np.sqrt((n_bins - 1) / n_bins * ((jk - jk.mean()) ** 2).sum())
    return float(full), float(err)
