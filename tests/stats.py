"""Binning (blocking) estimates of the mean and its standard error for
correlated Monte Carlo series."""
import numpy as np


def binned_mean(x, n_bins=50):
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // n_bins) * n_bins
    bins = x[:n].reshape(n_bins, -1).mean(axis=1)
    return float(bins.mean()), float(bins.std(ddof=1) / np.sqrt(n_bins))


def assert_within(estimate, error, exact, nsigma=4.0, floor=0.0, what=""):
    dev = abs(estimate - exact)
    assert dev <= nsigma * error + floor, (
        f"{what}: {estimate} +- {error} vs exact {exact} ({dev / max(error, 1e-300):.2f} sigma)")
