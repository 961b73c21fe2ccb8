"""The learned diagonal mass: training pipeline and the sampler that uses it.

Control flow only - every arithmetic step runs in librsv's kernels:
  1. run the plain (identity-mass) sampler and fold its h snapshots into
     per-site Welford moments (rsv_hmc_chain + rsv_welford_update);
  2. target log(1/Var(h_t)), its mean over the sites (the log of the output
     scale s) and the frozen posterior mean hbar (rsv_welford_target);
  3. standardised features from hbar, y, lnRV, theta (rsv_mass_features);
  4. Adam training of the BF16 MLP (rsv_mlp_train);
  5. inverse mass 1/m_t for every site (rsv_mlp_mass), m_t clamped to
     [1/s_u^2, diagonal of the Hessian of S at hbar].
The mass is a function of the frozen hbar only, so HMC with it stays exact.

The sampler that uses it (`MassSampler`) runs the chain in windows of
trajectories and falls back for good to the plain identity-mass sampler (its
own step size and trajectory length) when a window's acceptance rate is below
0.6 (checked while the next window runs, so the switch comes one window
later).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import rsv

NF, NH = 20, 32


def glorot_params(seed: int = 0) -> np.ndarray:
    """Initial FP32 parameter vector: Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)

    def glorot(o, i):
        lim = np.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, (o, i))
    W1, W2, W3 = glorot(NH, NF), glorot(NH, NH), glorot(1, NH)[0]
    return np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), W3,
                           np.zeros(1)]).astype(np.float32)


def collect_moments(ctx, h, y, lnrv, theta_dev, n_snap: int, n_md: int, dtau: float,
                    prec="mixed", seed: int = 0, traj0: int = 0, segment: int = 100,
                    update_theta: bool = False):
    """Run n_snap trajectories of the plain sampler from h (in place) and return
    the running per-site (mean, M2, count) of h over them."""
    T = h.numel()
    mean = torch.zeros(T, dtype=torch.float64, device=h.device)
    m2 = torch.zeros(T, dtype=torch.float64, device=h.device)
    snaps = torch.empty(segment, T, dtype=torch.float32, device=h.device)
    count, done = 0, 0
    while done < n_snap:
        k = min(segment, n_snap - done)
        view = snaps[:k]
        rsv.rsv_hmc_chain(ctx, h, y, lnrv, theta_dev, n_md, dtau, k, prec=prec, seed=seed,
                          traj0=traj0 + done, snaps=view, thin=1, update_theta=update_theta)
        count = rsv.rsv_welford_update(ctx, view, count, mean, m2)
        done += k
    return mean, m2, count


@dataclass
class TrainedMass:
    minv: torch.Tensor
    params: torch.Tensor
    log_scale: torch.Tensor
    losses: torch.Tensor
    target: torch.Tensor
    hbar: torch.Tensor
    features: torch.Tensor


def train_mass(ctx, y, lnrv, theta, mean, m2, count: int, steps: int = 2000, batch: int = 4096,
               lr: float = 1e-3, seed: int = 0, init_seed: int = 0) -> TrainedMass:
    """Steps 2-5: target, features, Adam training, inverse mass."""
    T = y.numel()
    hbar = torch.empty(T, dtype=torch.float64, device=y.device)
    log_s = torch.empty(1, dtype=torch.float32, device=y.device)
    target = rsv.rsv_welford_target(ctx, mean, m2, count, hbar_out=hbar, log_scale_out=log_s)
    feat, _ = rsv.rsv_mass_features(ctx, y, lnrv, hbar, theta)
    params = torch.tensor(glorot_params(init_seed), device=y.device)
    am = torch.zeros_like(params)
    av = torch.zeros_like(params)
    losses = torch.empty(max(steps, 1), dtype=torch.float32, device=y.device)
    rsv.rsv_mlp_train(ctx, feat, target, params, am, av, 0, steps, batch, seed, lr,
                      loss_out=losses if steps else None, log_scale=log_s)
    minv = rsv.rsv_mlp_mass(ctx, feat, params, y, hbar, theta, log_scale=log_s)
    return TrainedMass(minv=minv, params=params, log_scale=log_s, losses=losses[:steps],
                       target=target,
                       hbar=hbar, features=feat)


LADDER = (0.5, 0.4, 0.3, 0.25, 0.2, 0.15, 0.12, 0.1, 0.08, 0.07, 0.06, 0.05, 0.045, 0.04,
          0.035, 0.03, 0.025, 0.02, 0.015, 0.01)


def tune_step(ctx, h, y, lnrv, theta_dev, minv, length: float, prec="mixed",
              ladder=LADDER, n_try: int = 40, target_acc: float = 0.8, seed: int = 99):
    """Largest step of the ladder whose acceptance over n_try trajectories (of
    length ~ `length`) reaches target_acc; returns (dtau, n_md).  h is not
    modified."""
    acc = torch.empty(n_try, dtype=torch.int32, device=h.device)
    th = theta_dev.clone()
    for dt in ladder:
        n_md = max(1, int(round(length / dt)))
        hh = h.clone()
        rsv.rsv_hmc_chain(ctx, hh, y, lnrv, th, n_md, dt, n_try, prec=prec, minv=minv,
                          seed=seed, accept_out=acc)
        if float(acc.float().mean()) >= target_acc:
            return dt, n_md
    dt = ladder[-1]
    return dt, max(1, int(round(length / dt)))


@dataclass
class MassSampler:
    """Chain with the learned mass; identity-mass fallback below 0.6 acceptance."""
    ctx: rsv.Context
    minv: torch.Tensor
    dtau: float
    n_md: int
    plain_dtau: float
    plain_n_md: int
    window: int = 100
    prec: str = "mixed"
    fell_back: bool = False
    history: list = field(default_factory=list)
    md_steps: int = 0   # leapfrog steps run so far (per site)
    _pin: list = field(default_factory=list)  # two pinned host scalars (window rates)

    def run(self, h, y, lnrv, theta_dev, n_traj: int, seed: int, traj0: int = 0, snaps=None,
            theta_out=None, accept_out=None, update_theta: bool = True):
        T = h.numel()
        done = 0
        # a window's acceptance is read back without waiting for it: the
        # previous window's is checked while this one runs (so a collapse
        # switches to the plain sampler one window later, and the stream
        # never waits on the host between windows)
        pending = None
        if not self._pin:
            self._pin = [torch.empty((), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        slot = 0
        while done < n_traj:
            k = min(self.window, n_traj - done)
            acc = (accept_out[done:done + k] if accept_out is not None
                   else torch.empty(k, dtype=torch.int32, device=h.device))
            sn = snaps[done:done + k] if snaps is not None else None
            tho = theta_out[done:done + k] if theta_out is not None else None
            if self.fell_back:
                rsv.rsv_hmc_chain(self.ctx, h, y, lnrv, theta_dev, self.plain_n_md,
                                  self.plain_dtau, k, prec=self.prec, seed=seed,
                                  traj0=traj0 + done, snaps=sn, thin=1, theta_out=tho,
                                  accept_out=acc, update_theta=update_theta)
                self.md_steps += k * self.plain_n_md
            else:
                rsv.rsv_hmc_chain(self.ctx, h, y, lnrv, theta_dev, self.n_md, self.dtau, k,
                                  prec=self.prec, minv=self.minv, seed=seed, traj0=traj0 + done,
                                  snaps=sn, thin=1, theta_out=tho, accept_out=acc,
                                  update_theta=update_theta)
                self.md_steps += k * self.n_md
                host = self._pin[slot]
                slot ^= 1
                host.copy_(acc.float().mean(), non_blocking=True)
                ev = torch.cuda.Event()
                ev.record()
                prev, pending = pending, (ev, host)
                if prev is not None:
                    self._check(prev)
            done += k
        if pending is not None:
            self._check(pending)
        return h

    def _check(self, p):
        ev, host = p
        ev.synchronize()
        rate = float(host)
        self.history.append(rate)
        if rate < 0.6:
            self.fell_back = True
