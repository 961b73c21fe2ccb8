"""Independent references for the linear-Gaussian sub-case (test helpers).

With y_t = 0 the return equation (1) drops out of f except for its h_t/2 term,
and the posterior of h given (theta, lnRV) is exactly Gaussian.  Completing the
square, h_t/2 + (c_t - h_t)^2/(2 s_u^2) = (z_t - h_t)^2/(2 s_u^2) + const with
z_t = c_t - s_u^2/2, c_t = lnRV_t - xi.  So the posterior is that of the linear
state-space model
    x_{t+1} = phi x_t + eta_t,  x_1 ~ N(0, s_eta^2/(1-phi^2)),  z_t - mu = x_t + u_t,
which two textbook methods solve exactly:
  * a Kalman filter with Rauch-Tung-Striebel smoother (smoothed means/variances);
  * the tridiagonal posterior precision Q and linear term b, solved by the
    Thomas algorithm for the mean and a two-sided recurrence for diag(Q^-1).
Neither shares arithmetic with the oracle; they pin its action and force.
"""
from __future__ import annotations

import numpy as np


def rts_smoother(lnrv, theta):
    phi, mu, xi, se2, su2 = theta
    z = np.asarray(lnrv, dtype=np.float64) - xi - 0.5 * su2 - mu
    T = len(z)
    mp = np.empty(T); Pp = np.empty(T)   # predicted
    mf = np.empty(T); Pf = np.empty(T)   # filtered
    m, P = 0.0, se2 / (1.0 - phi * phi)
    for t in range(T):
        if t > 0:
            m, P = phi * mf[t - 1], phi * phi * Pf[t - 1] + se2
        mp[t], Pp[t] = m, P
        K = P / (P + su2)
        mf[t] = m + K * (z[t] - m)
        Pf[t] = (1.0 - K) * P
    ms = mf.copy(); Ps = Pf.copy()
    for t in range(T - 2, -1, -1):
        G = Pf[t] * phi / Pp[t + 1]
        ms[t] = mf[t] + G * (ms[t + 1] - mp[t + 1])
        Ps[t] = Pf[t] + G * G * (Ps[t + 1] - Pp[t + 1])
    return ms + mu, Ps


def tridiag_posterior(lnrv, theta):
    """Precision Q (diag d, off-diag o) and linear term b of the Gaussian
    posterior of h, mean = Q^-1 b by Thomas, var = diag(Q^-1) by recurrences."""
    phi, mu, xi, se2, su2 = theta
    c = np.asarray(lnrv, dtype=np.float64) - xi
    T = len(c)
    d = np.full(T, (1.0 + phi * phi) / se2 + 1.0 / su2)
    if T == 1:
        d[0] = (1.0 - phi * phi) / se2 + 1.0 / su2
    else:
        d[0] = d[-1] = 1.0 / se2 + 1.0 / su2
    o = np.full(max(T - 1, 0), -phi / se2)
    # linear term: from (c - h)^2/(2 su2) -> c/su2; from h/2 -> -1/2;
    # from the AR quadratic in x = h - mu -> mu * (row sums of the AR precision)
    ar_row = d - 1.0 / su2
    ar_row[:-1] += o
    ar_row[1:] += o
    b = c / su2 - 0.5 + mu * ar_row
    # Thomas algorithm for Q m = b
    cp = np.empty(max(T - 1, 0)); dp = np.empty(T)
    den = d[0]
    dp[0] = b[0] / den
    for t in range(T - 1):
        cp[t] = o[t] / den
        den = d[t + 1] - o[t] * cp[t]
        dp[t + 1] = (b[t + 1] - o[t] * dp[t]) / den
    m = dp.copy()
    for t in range(T - 2, -1, -1):
        m[t] = dp[t] - cp[t] * m[t + 1]
    # diag of the inverse: forward/backward pivots (Usmani-type recurrences)
    D = np.empty(T); E = np.empty(T)
    D[0] = d[0]
    for t in range(1, T):
        D[t] = d[t] - o[t - 1] ** 2 / D[t - 1]
    E[T - 1] = d[T - 1]
    for t in range(T - 2, -1, -1):
        E[t] = d[t] - o[t] ** 2 / E[t + 1]
    var = 1.0 / (D + E - d)
    return m, var, (d, o, b)
