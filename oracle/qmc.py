"""Sample statistics of the paper's QMC experiments (section 4, tests A1-A3;
test infrastructure only: nothing on the product path imports this module).

  quantile     the sample quantile, Hyndman and Fan's definition 7 (linear
               interpolation between order statistics at h = (n - 1) p),
               written out with a sort
  exceedance   P(c > threshold) per cell as the fraction of samples above it
  replicate_estimate
               mean of R independent randomised-QMC estimates and its
               standard error sqrt(var / R)
"""
from __future__ import annotations

import math

import numpy as np


def quantile(samples, p):
    """Sample quantile of 1-D `samples` at probability p in [0, 1]: with
    x_(0) <= ... <= x_(n-1) sorted, h = (n - 1) p, the value
    x_(floor h) + (h - floor h) (x_(floor h + 1) - x_(floor h))."""
    x = sorted(float(v) for v in samples)
    n = len(x)
    if n == 0:
        raise ValueError("no samples")
    h = (n - 1) * p
    k = int(math.floor(h))
    if k >= n - 1:
        return x[n - 1]
    return x[k] + (h - k) * (x[k + 1] - x[k])


def exceedance(c_samples, threshold):
    """Fraction of samples with c > threshold, per cell: c_samples [n, ...]."""
    c = np.asarray(c_samples, dtype=np.float64)
    return np.sum(c > threshold, axis=0) / c.shape[0]


def replicate_estimate(estimates):
    """Mean of R replicate estimates [R, ...] and its standard error."""
    e = np.asarray(estimates, dtype=np.float64)
    R = e.shape[0]
    mean = e.sum(axis=0) / R
    if R < 2:
        return mean, np.full(mean.shape, np.nan)
    var = ((e - mean) ** 2).sum(axis=0) / (R - 1)
    return mean, np.sqrt(var / R)
