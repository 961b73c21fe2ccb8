"""Seeded synthetic inputs for the RSV model (eqs. (1)-(3) of arXiv:1603.08114).

This module only draws data: it simulates the generative model and holds none
of the inference arithmetic (action, force, leapfrog, dH, Metropolis).  Both the
CUDA path and the CPU oracle take their inputs from here.

Draw order for one series (numpy ``default_rng(seed)``):
  h_1 ~ N(mu, s_eta^2 / (1 - phi^2)); eta_1..T-1 ~ N(0, s_eta^2);
  eps_1..T ~ N(0, 1); u_1..T ~ N(0, s_u^2);
  h_{t+1} = mu + phi (h_t - mu) + eta_t;  y_t = e^{h_t/2} eps_t;
  lnRV_t = xi + h_t + u_t.
The chain starts from h^(0)_t = lnRV_t - xi (the paper does not say where it
starts).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

#: theta of the fixed-parameter workloads: (phi, mu, xi, s_eta^2, s_u^2)
THETA_STD = (0.95, -0.5, -0.2, 0.05, 0.1)
#: theta of the 2^22-site mixed-precision workload
THETA_LARGE = (0.97, -0.5, -0.2, 0.03, 0.1)


@dataclass
class Series:
    h_true: np.ndarray
    y: np.ndarray
    lnrv: np.ndarray
    theta: tuple
    h0: np.ndarray  # initial chain state lnRV - xi


def _ar1(x0: float, eta: np.ndarray, phi: float) -> np.ndarray:
    """x_1 = x0, x_{t+1} = phi x_t + eta_t (the latent recursion of eq. (3))."""
    T = len(eta) + 1
    x = np.empty(T)
    x[0] = x0
    if T > 1:
        try:
            from scipy.signal import lfilter
            drive = np.concatenate(([x0], eta))
            x = lfilter([1.0], [1.0, -phi], drive)
        except ImportError:  # pragma: no cover - scipy is present on both machines
            for t in range(T - 1):
                x[t + 1] = phi * x[t] + eta[t]
    return x


def rsv_series(T: int, theta=THETA_STD, seed: int = 0) -> Series:
    """One synthetic RSV series of length T (eqs. (1)-(3))."""
    phi, mu, xi, se2, su2 = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    h1 = rng.normal(mu, np.sqrt(se2 / (1.0 - phi * phi)))
    eta = rng.normal(0.0, np.sqrt(se2), T - 1)
    eps = rng.normal(0.0, 1.0, T)
    u = rng.normal(0.0, np.sqrt(su2), T)
    h = _ar1(h1 - mu, eta, phi) + mu
    y = np.exp(h / 2.0) * eps
    lnrv = xi + h + u
    return Series(h_true=h, y=y, lnrv=lnrv, theta=(phi, mu, xi, se2, su2), h0=lnrv - xi)


#: leverage of the RSV-with-leverage workloads: corr(eps_t, eta_t), negative as
#: for equity returns (a fall in price raises the next volatility)
RHO_STD = -0.4


def rsv_series_leverage(T: int, theta=THETA_STD, rho: float = RHO_STD, seed: int = 0) -> Series:
    """One synthetic series of the RSV model with leverage: eqs. (1)-(3) with
    corr(eps_t, eta_t) = rho.  Draw order: h_1 ~ N(mu, s_eta^2 / (1 - phi^2));
    eps_1..T ~ N(0, 1); z_1..T-1 ~ N(0, 1); u_1..T ~ N(0, s_u^2);
    eta_t = s_eta (rho eps_t + sqrt(1 - rho^2) z_t)."""
    phi, mu, xi, se2, su2 = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    h1 = rng.normal(mu, np.sqrt(se2 / (1.0 - phi * phi)))
    eps = rng.normal(0.0, 1.0, T)
    z = rng.normal(0.0, 1.0, T - 1)
    u = rng.normal(0.0, np.sqrt(su2), T)
    eta = np.sqrt(se2) * (rho * eps[:-1] + np.sqrt(1.0 - rho * rho) * z)
    h = _ar1(h1 - mu, eta, phi) + mu
    y = np.exp(h / 2.0) * eps
    lnrv = xi + h + u
    return Series(h_true=h, y=y, lnrv=lnrv, theta=(phi, mu, xi, se2, su2), h0=lnrv - xi)


def standard_normals(n: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) draws (momenta passed in explicitly by parity tests)."""
    return np.random.default_rng(seed).standard_normal(n)


def log_uniforms(n: int, seed: int) -> np.ndarray:
    """Seeded ln u, u ~ U(0,1) (Metropolis uniforms passed in explicitly)."""
    return np.log(np.random.default_rng(seed).random(n))


@dataclass
class Batch:
    """Many independent series packed end to end: series s occupies
    [offsets[s], offsets[s+1]) of y, lnrv and h0; theta is (n, 5)."""
    offsets: np.ndarray
    y: np.ndarray
    lnrv: np.ndarray
    h0: np.ndarray
    h_true: np.ndarray
    theta: np.ndarray


def rsv_batch(n_series: int, T_lo: int, T_hi: int, seed: int = 2) -> Batch:
    """Batched workload: T ~ U{T_lo..T_hi}; per-series theta with
    phi ~ U(0.85, 0.99), mu ~ N(-0.5, 0.3), xi ~ N(-0.2, 0.1),
    s_eta^2 ~ U(0.02, 0.1), s_u^2 ~ U(0.05, 0.2) (second argument of N read as
    a standard deviation)."""
    rng = np.random.default_rng(seed)
    Ts = rng.integers(T_lo, T_hi + 1, n_series)
    th = np.stack([rng.uniform(0.85, 0.99, n_series), rng.normal(-0.5, 0.3, n_series),
                   rng.normal(-0.2, 0.1, n_series), rng.uniform(0.02, 0.1, n_series),
                   rng.uniform(0.05, 0.2, n_series)], axis=1)
    offsets = np.zeros(n_series + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Ts)
    N = int(offsets[-1])
    y = np.empty(N)
    lnrv = np.empty(N)
    h_true = np.empty(N)
    for s in range(n_series):
        ser = rsv_series(int(Ts[s]), tuple(th[s]), seed=int(rng.integers(0, 2**62)))
        a, b = offsets[s], offsets[s + 1]
        y[a:b], lnrv[a:b], h_true[a:b] = ser.y, ser.lnrv, ser.h_true
    h0 = lnrv - np.repeat(th[:, 2], Ts)
    return Batch(offsets=offsets, y=y, lnrv=lnrv, h0=h0, h_true=h_true, theta=th)
