"""Small statistics helpers for the sampling tests (block averaging)."""
import numpy as np


def block_mean_sigma(series, nblocks=20):
    """Mean of a time series and the standard error from nblocks block means."""
    a = np.asarray(series, dtype=np.float64)
    n = (len(a) // nblocks) * nblocks
    b = a[len(a) - n:].reshape(nblocks, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nblocks))
