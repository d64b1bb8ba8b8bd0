"""Binning and jackknife error analysis (test infrastructure).

The paper quotes 1-sigma errors from a jackknife analysis (Sec. 5).  Here a
time series of per-update measurements is cut into bins longer than the
autocorrelation time; bin means give the standard error, and ratios of means
(the correlation length) get jackknife errors.
"""
import numpy as np


def binned(x, nbins=50):
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // nbins
    return x[: m * nbins].reshape(nbins, m).mean(axis=1)


def mean_err(x, nbins=50):
    b = binned(x, nbins)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(len(b)))


def jackknife(f, *series, nbins=50):
    """Jackknife estimate and error of f(mean(a), mean(b), ...)."""
    bins = [binned(s, nbins) for s in series]
    n = len(bins[0])
    tot = [b.sum() for b in bins]
    full = f(*[t / n for t in tot])
    jk = np.array([f(*[(t - b[i]) / (n - 1) for t, b in zip(tot, bins)]) for i in range(n)])
    err = np.sqrt((n - 1) / n * ((jk - jk.mean()) ** 2).sum())
    return float(full), float(err)


def xi_second_moment(L):
    """xi = (L / 2 pi) sqrt(chi(pi) / chi(pi + 2 pi / L) - 1)."""
    def f(chi_s, chi_q):
        return L / (2 * np.pi) * np.sqrt(max(chi_s / chi_q - 1.0, 0.0))
    return f


def xi_tau(beta):
    """xi_tau = (beta / 2 pi) sqrt(chi(pi, 0) / chi(pi, 2 pi / beta) - 1): the
    imaginary-time second moment (Sec. 5); the gap is 1 / xi_tau."""
    def f(chi_s, chi_w):
        return beta / (2 * np.pi) * np.sqrt(max(chi_s / chi_w - 1.0, 0.0))
    return f


def within_sigma(value, err, ref, nsigma=3.0, ref_err=0.0):
    return abs(value - ref) <= nsigma * np.sqrt(err ** 2 + ref_err ** 2)
