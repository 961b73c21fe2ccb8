"""Pins of the oracle's RSV model with leverage, corr(eps_t, eta_t) = rho (the
model of the RSV reference the paper cites in Sec. 2), against things other
than itself (CPU only): the joint density of (y, lnRV, h) written with scipy's
bivariate normal, central finite differences, the plain model at rho = 0,
reversibility and the second-order energy error of the leapfrog, and posterior
moments of a tiny series by quadrature."""
import numpy as np
import pytest

import oracle
from oracle import stats
from paper_1603_08114_gb300 import synth

TH = synth.THETA_STD


def _log_joint(h, y, lnrv, th, rho):
    """ln p(y, lnRV, h | theta, rho) from the generative model: h_1 stationary,
    (eps_t, eta_t) bivariate normal with covariance [[1, rho s], [rho s, s^2]]
    for t < T, eps_T standard normal, lnRV_t | h_t normal; the change of
    variables (y_t, h_{t+1}) -> (eps_t, eta_t) has Jacobian e^{-h_t/2}."""
    from scipy.stats import multivariate_normal, norm
    phi, mu, xi, se2, su2 = th
    se = np.sqrt(se2)
    T = len(h)
    eps = y * np.exp(-h / 2)
    lp = norm.logpdf(h[0], mu, np.sqrt(se2 / (1 - phi * phi)))
    lp += np.sum(norm.logpdf(lnrv, xi + h, np.sqrt(su2)))
    if T > 1:
        eta = (h[1:] - mu) - phi * (h[:-1] - mu)
        cov = np.array([[1.0, rho * se], [rho * se, se2]])
        lp += np.sum(multivariate_normal(mean=[0.0, 0.0], cov=cov).logpdf(
            np.stack([eps[:-1], eta], axis=1)))
    lp += norm.logpdf(eps[-1])
    lp += np.sum(-h / 2)
    return lp


@pytest.mark.parametrize("rho", [-0.6, 0.35])
@pytest.mark.parametrize("T", [1, 2, 5, 40])
def test_action_is_minus_log_joint_density(T, rho):
    """S(h) - S(h') = -(ln p(h) - ln p(h')): constants cancel in the difference."""
    s = synth.rsv_series_leverage(T, TH, rho, seed=T)
    rng = np.random.default_rng(11)
    th = TH + (rho,)
    for _ in range(3):
        h1 = s.h_true + 0.4 * rng.standard_normal(T)
        h2 = s.h_true + 0.4 * rng.standard_normal(T)
        dS = oracle.action(h1, s.y, s.lnrv, th) - oracle.action(h2, s.y, s.lnrv, th)
        dL = _log_joint(h2, s.y, s.lnrv, TH, rho) - _log_joint(h1, s.y, s.lnrv, TH, rho)
        assert abs(dS - dL) < 1e-9 * max(1.0, abs(dS))


def test_leverage_sign_matters():
    """A wrong sign of rho would fail the density pin: the action differs between
    rho and -rho on data with returns (it is even in rho only if y = 0)."""
    s = synth.rsv_series_leverage(20, TH, -0.5, seed=2)
    a = oracle.action(s.h_true, s.y, s.lnrv, TH + (-0.5,))
    b = oracle.action(s.h_true, s.y, s.lnrv, TH + (0.5,))
    assert abs(a - b) > 1e-3
    z = np.zeros(20)
    assert oracle.action(s.h_true, z, s.lnrv, TH + (-0.5,)) == pytest.approx(
        oracle.action(s.h_true, z, s.lnrv, TH + (0.5,)), rel=1e-14)


@pytest.mark.parametrize("rho", [-0.7, 0.5])
@pytest.mark.parametrize("T", [1, 2, 3, 9])
def test_force_matches_finite_differences(T, rho):
    s = synth.rsv_series_leverage(T, TH, rho, seed=T + 4)
    th = TH + (rho,)
    h = s.h_true + 0.3 * np.random.default_rng(5).standard_normal(T)
    F = oracle.force(h, s.y, s.lnrv, th)
    eps = 1e-5
    fd = np.empty(T)
    for t in range(T):
        hp, hm = h.copy(), h.copy()
        hp[t] += eps
        hm[t] -= eps
        fd[t] = (oracle.action(hp, s.y, s.lnrv, th) - oracle.action(hm, s.y, s.lnrv, th)) / (2 * eps)
    assert np.max(np.abs(F - fd) / np.maximum(np.abs(F), 1.0)) < 1e-7


def test_rho_zero_is_the_plain_model():
    """rho = 0 reproduces the action of eqs. (1)-(3) written out with numpy."""
    T = 30
    s = synth.rsv_series(T, TH, seed=3)
    phi, mu, xi, se2, su2 = TH
    h, x = s.h_true, s.h_true - mu
    S = (np.sum(h / 2 + 0.5 * s.y ** 2 * np.exp(-h) + (s.lnrv - xi - h) ** 2 / (2 * su2))
         + (1 - phi ** 2) * x[0] ** 2 / (2 * se2) + np.sum((x[1:] - phi * x[:-1]) ** 2) / (2 * se2))
    assert oracle.action(h, s.y, s.lnrv, TH + (0.0,)) == pytest.approx(S, rel=1e-12)


def test_leapfrog_reversible_and_second_order_under_leverage():
    T = 64
    s = synth.rsv_series_leverage(T, TH, -0.4, seed=9)
    th = TH + (-0.4,)
    p = synth.standard_normals(T, 4)
    h1, p1 = oracle.leapfrog(s.h_true, p, s.y, s.lnrv, th, 20, 0.02)
    h2, p2 = oracle.leapfrog(h1, -p1, s.y, s.lnrv, th, 20, 0.02)
    assert np.max(np.abs(h2 - s.h_true)) < 1e-11
    assert np.max(np.abs(p2 + p)) < 1e-10
    dH = []
    for dt in (0.02, 0.01):
        n = int(round(0.4 / dt))
        hh, pp = oracle.leapfrog(s.h_true, p, s.y, s.lnrv, th, n, dt)
        dH.append(oracle.delta_H(s.h_true, p, hh, pp, s.y, s.lnrv, th))
    assert 3.0 < abs(dH[0] / dH[1]) < 5.5


def test_theta_update_refused_under_leverage():
    s = synth.rsv_series_leverage(10, TH, -0.4, seed=1)
    with pytest.raises(ValueError):
        oracle.chain(s.h_true, s.y, s.lnrv, TH + (-0.4,), 5, 0.05, seed=1, n_traj=2,
                     update_theta=True)
    with pytest.raises(ValueError):
        oracle.gibbs_theta(s.h_true, s.lnrv, TH + (-0.4,), 1, 0, 0)


@pytest.mark.slow
def test_T2_posterior_by_quadrature_under_leverage():
    """HMC with leverage samples exp(-S): posterior means and variances of a
    two-site series against a 2-D quadrature of exp(-S) written with the
    density pinned above."""
    rho = -0.6
    th = TH + (rho,)
    y = np.array([-1.1, 0.7])
    lnrv = np.array([-0.3, -0.9])
    g = np.linspace(-5.0, 3.5, 401)
    H1, H2 = np.meshgrid(g, g, indexing="ij")
    lp = np.empty_like(H1)
    for i in range(len(g)):
        for j in range(len(g)):
            lp[i, j] = -oracle.action(np.array([H1[i, j], H2[i, j]]), y, lnrv, th)
    w = np.exp(lp - lp.max())
    w /= w.sum()
    m = np.array([np.sum(H1 * w), np.sum(H2 * w)])
    v = np.array([np.sum((H1 - m[0]) ** 2 * w), np.sum((H2 - m[1]) ** 2 * w)])
    r = oracle.chain(m.copy(), y, lnrv, th, n_md=8, dtau=0.08, seed=31, n_traj=20000, thin=1)
    x = r["snaps"]
    for k in range(2):
        assert abs(x[:, k].mean() - m[k]) < 3.5 * stats.batch_means_mcse(x[:, k])
        assert abs(x[:, k].var() - v[k]) < 3.5 * stats.batch_means_mcse((x[:, k] - m[k]) ** 2)
