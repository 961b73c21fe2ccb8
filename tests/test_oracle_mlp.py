"""Pins of the FP64 learned-mass reference (CPU): finite differences of the
loss, the closed-form first Adam step, BF16 rounding, feature layout,
standardisation, minibatch indices."""
import numpy as np
import pytest

from oracle import mlp
from paper_1603_08114_gb300 import synth


def _data(T=300, seed=0):
    s = synth.rsv_series(T, synth.THETA_STD, seed=seed)
    hbar = s.h_true + 0.01 * np.sin(np.arange(T))
    F = mlp.features_raw(s.y, s.lnrv, hbar, s.theta)
    Fn, m, inv = mlp.standardize(F)
    target = -np.log(0.02 + 0.01 * np.cos(np.arange(T)) ** 2)
    return Fn, target, s, hbar


def test_bf16_rounding_ties_to_even():
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                   # tie -> even
    assert mlp.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7   # above the tie
    assert mlp.bf16(1.0 + 2.0 ** -7 + 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert mlp.bf16(-3.0) == -3.0


def test_loss_gradient_matches_finite_differences():
    Fn, target, _, _ = _data()
    P = mlp.init_params(3)
    L, G = mlp.loss_and_grads(P, Fn, target, bf=False)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            Pp = {kk: v.copy() for kk, v in P.items()}
            Pm = {kk: v.copy() for kk, v in P.items()}
            Pp[k].reshape(-1)[i] += eps
            Pm[k].reshape(-1)[i] -= eps
            fd = (mlp.loss_and_grads(Pp, Fn, target, bf=False)[0]
                  - mlp.loss_and_grads(Pm, Fn, target, bf=False)[0]) / (2 * eps)
            assert abs(fd - G[k].reshape(-1)[i]) <= 1e-6 * max(1.0, abs(fd)), (k, i)


def test_first_adam_step_is_lr_times_sign():
    P = mlp.init_params(1)
    G = {k: np.where(np.arange(v.size).reshape(v.shape) % 3 == 0, 0.0, (-1.0) ** np.arange(v.size).reshape(v.shape) * 0.37)
         for k, v in P.items()}
    P0 = {k: v.copy() for k, v in P.items()}
    opt = mlp.Adam(P, lr=1e-3)
    opt.step(P, G)
    for k in P:
        step = P0[k] - P[k]
        exp = 1e-3 * G[k] / (np.abs(G[k]) + 1e-8)
        assert np.allclose(step, exp, rtol=1e-12, atol=1e-15)


def test_features_layout_and_standardisation():
    T = 12
    s = synth.rsv_series(T, synth.THETA_STD, seed=1)
    hbar = np.arange(T) * 0.1 - 0.5
    F = mlp.features_raw(s.y, s.lnrv, hbar, s.theta)
    assert F.shape == (T, 20)
    assert np.allclose(F[:, 0], s.y ** 2) and np.allclose(F[:, 1], s.lnrv)
    assert F[0, 2] == 0 and F[0, 5] == 0 and F[0, 6] == hbar[0] and F[0, 10] == hbar[4]
    assert F[T - 1, 10] == 0 and F[T - 1, 6] == hbar[T - 1]
    assert F[0, 16] == 1 and F[T - 1, 16] == 1 and F[3, 16] == 0
    phi, mu, xi, se2, su2 = s.theta
    assert np.allclose(F[:, 17], (1 + phi * phi) / se2) and np.allclose(F[:, 18], 1 / su2)
    assert np.allclose(F[:, 19], 0.5 * s.y ** 2 * np.exp(-hbar))
    Fn, m, inv = mlp.standardize(F)
    varying = F.std(0) > 1e-12 * np.maximum(1.0, np.abs(F.mean(0)))
    assert np.allclose(Fn[:, varying].mean(0), 0, atol=1e-12)
    assert np.allclose(Fn[:, varying].std(0), 1, atol=1e-12)
    assert np.all(Fn[:, ~varying] == 0)


def test_batch_indices_cover_range_uniformly():
    T, B = 1000, 4096
    idx = np.concatenate([mlp.batch_indices(7, st, T, B) for st in range(3)])
    assert idx.min() >= 0 and idx.max() < T
    counts = np.bincount(idx, minlength=T)
    from scipy import stats as sps
    assert sps.chisquare(counts).pvalue > 1e-3


def test_training_reduces_loss_fp64():
    Fn, target, _, _ = _data(T=512)
    P = mlp.init_params(0)
    opt = mlp.Adam(P, lr=1e-2)
    L0 = mlp.loss_and_grads(P, Fn, target)[0]
    for _ in range(200):
        L, G = mlp.loss_and_grads(P, Fn, target)
        opt.step(P, G)
    assert L < 0.2 * L0
