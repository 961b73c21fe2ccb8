"""FP64 reference of the learned diagonal mass (TEST INFRASTRUCTURE ONLY).

The paper has no learned part; this is the reference for the network the
library adds.  A site's mass is m_t = s (softplus(z_t) + eps_m) with z_t the output of a
20 -> 32 -> 32 -> 1 MLP (tanh hidden units) on 20 features of the site; it is
trained by Adam on the squared error between log m_t and the target
log(1 / Var(h_t)) estimated from sampler snapshots.  s is a fixed output scale
(log s = the mean of the target over the sites), so softplus works near unit
slope instead of the tanh layers saturating to reach precisions of O(30).

The CUDA path computes the matmuls in BF16 with FP32 accumulation.  To compare
like with like this reference applies BF16 rounding (round to nearest even) at
the same points - the matmul operands: features, weights of layers 1-2, the
hidden activation a1, and the back-propagated dz1/dz2 - and accumulates in
FP64.  With ``bf16=False`` it is the plain FP64 network (used by the
finite-difference pins).

Features of site t (20: the local data y_t^2 and lnRV_t, an 8-neighbour window of
the frozen posterior mean, theta, and position terms):
  0  y_t^2                      1  lnRV_t
  2..10  hbar_{t-4} .. hbar_{t+4} (frozen posterior mean of h; 0 past the ends)
  11..15 phi, mu, xi, s_eta^2, s_u^2
  16 edge proximity 2^-d, d = distance to the nearer end (1 at both ends)
  17 (1 + phi^2) / s_eta^2
  18 1 / s_u^2                  19 (y_t^2 / 2) e^{-hbar_t}
standardised per feature over the sites (mean 0, sd 1; constant features -> 0)
except the edge proximity, and clipped to [-8, 8].  At inference the mass is clamped
to [1/s_u^2, diagonal of the Hessian of S at hbar] (`mass_bounds`).
"""
from __future__ import annotations

import numpy as np

NF, NH = 20, 32
EPS_M = 1e-3


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features_raw(y, lnrv, hbar, theta):
    phi, mu, xi, se2, su2 = (float(v) for v in theta)
    T = len(y)
    F = np.zeros((T, NF))
    F[:, 0] = y * y
    F[:, 1] = lnrv
    for k in range(-4, 5):
        col = 2 + (k + 4)
        src = np.arange(T) + k
        ok = (src >= 0) & (src < T)
        F[ok, col] = hbar[src[ok]]
    F[:, 11:16] = [phi, mu, xi, se2, su2]
    d = np.minimum(np.arange(T), T - 1 - np.arange(T))
    F[:, 16] = 2.0 ** -np.minimum(d, 64).astype(np.float64)
    F[:, 17] = (1.0 + phi * phi) / se2
    F[:, 18] = 1.0 / su2
    F[:, 19] = 0.5 * y * y * np.exp(-hbar)
    return F


EDGE = 16      # the edge proximity 2^-d is left unstandardised
CLIP = 8.0     # standardised features are clipped to [-8, 8]


def standardize(F):
    """Per-feature mean and sd over the sites (columns with sd ~ 0 map to 0),
    except the edge proximity, which stays as is; then clip to [-CLIP, CLIP]."""
    m = F.mean(axis=0)
    sd = F.std(axis=0)
    inv = np.where(sd > 1e-12 * np.maximum(1.0, np.abs(m)), 1.0 / np.where(sd > 0, sd, 1), 0.0)
    m[EDGE] = 0.0
    inv[EDGE] = 1.0
    return np.clip((F - m) * inv, -CLIP, CLIP), m, inv


def mass_bounds(y, hbar, theta):
    """Interval the inferred mass is clamped to: from the observation precision
    1/s_u^2 (a floor of the posterior precision of h_t) to the diagonal of the
    Hessian of S at hbar, A_t/s_eta^2 + 1/s_u^2 + (y_t^2/2) e^{-hbar_t} with
    A_t = 1 + phi^2 inside, 1 at the two ends, 1 - phi^2 if T = 1."""
    phi, mu, xi, se2, su2 = (float(v) for v in theta)
    T = len(y)
    A = np.full(T, 1.0 + phi * phi)
    if T == 1:
        A[0] = 1.0 - phi * phi
    else:
        A[0] = A[-1] = 1.0
    lo = np.full(T, 1.0 / su2)
    hi = A / se2 + 1.0 / su2 + 0.5 * y * y * np.exp(-hbar)
    return lo, hi


def init_params(seed=0):
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)

    def glorot(o, i):
        lim = np.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, (o, i))
    return {"W1": glorot(NH, NF), "b1": np.zeros(NH), "W2": glorot(NH, NH), "b2": np.zeros(NH),
            "W3": glorot(1, NH)[0], "b3": np.zeros(1)}


def softplus(z):
    return np.logaddexp(0.0, z)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(P, Fn, bf=True, log_s=0.0):
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    f = r(Fn)
    z1 = f @ r(P["W1"]).T + P["b1"]
    a1 = np.tanh(z1)
    z2 = r(a1) @ r(P["W2"]).T + P["b2"]
    a2 = np.tanh(z2)
    z3 = a2 @ P["W3"] + P["b3"][0]
    u = softplus(z3) + EPS_M
    return dict(f=f, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, u=u, m=np.exp(log_s) * u)


def loss_and_grads(P, Fn, target, bf=True, log_s=0.0):
    """Mean squared error of log m against target and its gradients."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    c = forward(P, Fn, bf, log_s)
    B = len(target)
    lm = log_s + np.log(c["u"])
    L = np.mean((lm - target) ** 2)
    g3 = 2.0 * (lm - target) / B * sigmoid(c["z3"]) / c["u"]
    G = {"W3": c["a2"].T @ g3, "b3": np.array([g3.sum()])}
    dz2 = np.outer(g3, P["W3"]) * (1.0 - c["a2"] ** 2)
    G["W2"] = r(dz2).T @ r(c["a1"])
    G["b2"] = dz2.sum(axis=0)
    da1 = r(dz2) @ r(P["W2"])
    dz1 = da1 * (1.0 - c["a1"] ** 2)
    G["W1"] = r(dz1).T @ c["f"]
    G["b1"] = dz1.sum(axis=0)
    return L, G


class Adam:
    """Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
    w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, P, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in P.items()}
        self.v = {k: np.zeros_like(v) for k, v in P.items()}
        self.t = 0

    def step(self, P, G):
        self.t += 1
        for k in P:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * G[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * G[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            P[k] = P[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def batch_indices(seed, step, T, B):
    """Minibatch site indices of Adam step `step`: word w of Philox block
    (counter {b, step, 3, 0}, key {seed, 0}) gives index floor(hi32(w) * T / 2^32)."""
    import oracle
    out = np.empty(B, dtype=np.int64)
    for b in range((B + 3) // 4):
        w = oracle.philox4x64_10((b, step, 3, 0), (seed, 0))
        for i in range(4):
            k = 4 * b + i
            if k < B:
                out[k] = ((int(w[i]) >> 32) * T) >> 32
    return out


def welford_reference(X):
    """Two-pass mean and unbiased variance over the rows of X."""
    X = np.asarray(X, dtype=np.float64)
    m = X.mean(axis=0)
    return m, ((X - m) ** 2).sum(axis=0) / (X.shape[0] - 1)
