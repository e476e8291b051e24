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
