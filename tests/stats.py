"""Binned jackknife estimates of sign-weighted Monte Carlo averages."""
import numpy as np


def jackknife_ratio(records, col, nbins=40):
    """<O> = <sign*O>/<sign> from per-sweep records (col 0 = sign)."""
    n = (len(records) // nbins) * nbins
    r = records[:n].reshape(nbins, n // nbins, -1).mean(axis=1)
    num, den = r[:, col], r[:, 0]
    est = num.mean() / den.mean()
    jk = np.array([(num.sum() - num[b]) / (den.sum() - den[b]) for b in range(nbins)])
    err = np.sqrt((nbins - 1) / nbins * np.sum((jk - jk.mean()) ** 2))
    return est, err
