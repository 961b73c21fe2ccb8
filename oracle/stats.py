"""MCMC-output estimators used as references (TEST INFRASTRUCTURE ONLY).

- Geyer's initial monotone sequence estimator of the integrated
  autocorrelation time (C. J. Geyer, "Practical Markov chain Monte Carlo",
  Statistical Science 7, 1992): with normalised autocorrelations rho_k, form
  pair sums Gamma_m = rho_{2m} + rho_{2m+1}, stop at the first m with
  Gamma_m <= 0, make the retained sequence non-increasing, and take
  tau = -1 + 2 sum_m Gamma_m; ESS = n / tau.
- Batch-means Monte-Carlo standard error with floor(sqrt(n)) batches.
- Two-pass mean and variance (the definition the on-device Welford update must
  reproduce).
Autocovariances are the plain sums gamma_k = (1/n) sum_t (x_t - m)(x_{t+k} - m).
"""
from __future__ import annotations

import numpy as np


def autocov(x: np.ndarray, max_lag: int | None = None) -> np.ndarray:
    """gamma_k for k = 0..max_lag along axis 0 (plain sums, biased 1/n)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if max_lag is None:
        max_lag = n - 1
    d = x - x.mean(axis=0)
    out = np.empty((max_lag + 1,) + x.shape[1:])
    for k in range(max_lag + 1):
        out[k] = (d[: n - k] * d[k:]).sum(axis=0) / n
    return out


def ess_geyer(x: np.ndarray) -> np.ndarray:
    """Effective sample size along axis 0 by Geyer's initial monotone sequence."""
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    n = x.shape[0]
    g = autocov(x)
    out = np.empty(x.shape[1])
    for j in range(x.shape[1]):
        if g[0, j] <= 0.0:  # constant column: the chain never moved
            out[j] = 0.0
            continue
        rho = g[:, j] / g[0, j]
        tau_sum = 0.0
        prev = np.inf
        m = 0
        while 2 * m + 1 < n:
            G = rho[2 * m] + rho[2 * m + 1]
            if G <= 0.0:
                break
            G = min(G, prev)
            tau_sum += G
            prev = G
            m += 1
        tau = -1.0 + 2.0 * tau_sum
        tau = max(tau, 1.0 / np.log10(max(n, 10)))
        out[j] = n / tau
    return out[0] if squeeze else out


def batch_means_mcse(x: np.ndarray) -> np.ndarray:
    """Monte-Carlo standard error of the mean by batch means, floor(sqrt(n)) batches."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    b = max(int(np.floor(np.sqrt(n))), 2)
    L = n // b
    xb = x[: b * L].reshape((b, L) + x.shape[1:]).mean(axis=1)
    return np.sqrt(xb.var(axis=0, ddof=1) / b)


def mean_var(x: np.ndarray):
    """Two-pass mean and unbiased variance along axis 0."""
    x = np.asarray(x, dtype=np.float64)
    m = x.mean(axis=0)
    v = ((x - m) ** 2).sum(axis=0) / (x.shape[0] - 1)
    return m, v
