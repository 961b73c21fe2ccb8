"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names what fixes the expected value: a closed form, an independent
textbook algorithm (Kalman/RTS smoother, tridiagonal solve, quadrature), numpy's
own Philox, finite differences, or an exact property of the leapfrog of
eqs. (6)-(8) (reversibility, second-order energy error) or of the Metropolis
step of Sec. 3 (the Creutz identity <exp(-dH)> = 1).
"""
import numpy as np
import pytest

import oracle
from oracle import stats
from paper_1603_08114_gb300 import synth
from tests.kalman_pin import rts_smoother, tridiag_posterior

TH = synth.THETA_STD


def _series(T, seed=0, theta=TH):
    return synth.rsv_series(T, theta, seed)


# --------------------------------------------------------------------------
# gradient of S (eq. (7)) against central finite differences of S
# --------------------------------------------------------------------------
@pytest.mark.parametrize("T", [1, 2, 3, 7, 64])
def test_force_matches_finite_differences(T):
    s = _series(T, seed=T)
    rng = np.random.default_rng(5)
    h = s.h_true + 0.3 * rng.standard_normal(T)
    F = oracle.force(h, s.y, s.lnrv, TH)
    eps = 1e-5
    fd = np.empty(T)
    for t in range(T):
        hp, hm = h.copy(), h.copy()
        hp[t] += eps
        hm[t] -= eps
        fd[t] = (oracle.action(hp, s.y, s.lnrv, TH) - oracle.action(hm, s.y, s.lnrv, TH)) / (2 * eps)
    scale = np.maximum(np.abs(F), 1.0)
    assert np.max(np.abs(F - fd) / scale) < 1e-7


def test_action_matches_closed_form_sum():
    """S written term by term from eqs. (1)-(3) (independent vectorised numpy)."""
    T = 50
    s = _series(T, seed=3)
    phi, mu, xi, se2, su2 = TH
    h = s.h_true
    x = h - mu
    S = (np.sum(h / 2 + 0.5 * s.y ** 2 * np.exp(-h) + (s.lnrv - xi - h) ** 2 / (2 * su2))
         + (1 - phi ** 2) * x[0] ** 2 / (2 * se2) + np.sum((x[1:] - phi * x[:-1]) ** 2) / (2 * se2))
    assert abs(oracle.action(h, s.y, s.lnrv, TH) - S) < 1e-11 * abs(S)
    assert np.allclose(oracle.action_sites(h, s.y, s.lnrv, TH).sum(), S, rtol=1e-13)


# --------------------------------------------------------------------------
# linear-Gaussian sub-case: Kalman/RTS and tridiagonal solve pin S and dS/dh
# --------------------------------------------------------------------------
@pytest.mark.parametrize("T", [1, 2, 5, 300])
def test_gaussian_subcase_mode_and_hessian(T):
    s = _series(T, seed=11)
    y0 = np.zeros(T)
    m_kf, v_kf = rts_smoother(s.lnrv, TH)
    m_td, v_td, (d, o, b) = tridiag_posterior(s.lnrv, TH)
    # the two independent exact solvers agree
    assert np.max(np.abs(m_kf - m_td)) < 1e-12
    assert np.max(np.abs(v_kf - v_td) / v_td) < 1e-12
    # the posterior mean is the stationary point of S: dS/dh = 0 there
    F = oracle.force(m_kf, y0, s.lnrv, TH)
    assert np.max(np.abs(F)) < 1e-9
    # the Hessian of S is the precision Q: F(m + e_t) - F(m) is column t of Q
    for t in sorted({0, T // 2, T - 1}):
        e = np.zeros(T)
        e[t] = 1.0
        col = oracle.force(m_kf + e, y0, s.lnrv, TH) - F
        ref = np.zeros(T)
        ref[t] = d[t]
        if t > 0:
            ref[t - 1] = o[t - 1]
        if t + 1 < T:
            ref[t + 1] = o[t]
        assert np.max(np.abs(col - ref)) < 1e-9


@pytest.mark.slow
def test_gaussian_subcase_hmc_moments_match_smoother():
    """HMC chain (Philox momenta, Metropolis) reproduces the exact posterior
    mean and variance within 3 Monte-Carlo standard errors."""
    T = 40
    s = _series(T, seed=12)
    y0 = np.zeros(T)
    m_kf, v_kf = rts_smoother(s.lnrv, TH)
    r = oracle.chain(m_kf.copy(), y0, s.lnrv, TH, n_md=12, dtau=0.05, seed=77, n_traj=6000,
                     thin=1)
    x = r["snaps"][500:]
    mean = x.mean(axis=0)
    se = stats.batch_means_mcse(x)
    z = np.abs(mean - m_kf) / se
    assert np.mean(z < 3.0) > 0.95 and np.max(z) < 5.0
    var = x.var(axis=0, ddof=1)
    se_v = stats.batch_means_mcse((x - m_kf) ** 2)
    zv = np.abs(var - v_kf) / se_v
    assert np.mean(zv < 3.0) > 0.95 and np.max(zv) < 5.0


# --------------------------------------------------------------------------
# leapfrog properties (eqs. (6)-(8))
# --------------------------------------------------------------------------
def test_leapfrog_reversible():
    T = 2000
    s = _series(T, seed=0)
    p0 = synth.standard_normals(T, 1)
    h1, p1 = oracle.leapfrog(s.h0, p0, s.y, s.lnrv, TH, 50, 0.02)
    h2, p2 = oracle.leapfrog(h1, -p1, s.y, s.lnrv, TH, 50, 0.02)
    assert np.max(np.abs(h2 - s.h0)) < 1e-12
    assert np.max(np.abs(-p2 - p0)) < 1e-12


def test_leapfrog_energy_error_is_second_order():
    T = 500
    s = _series(T, seed=4)
    rng = np.random.default_rng(9)
    h0 = s.h_true.copy()
    p0 = rng.standard_normal(T)
    L = 0.32
    # asymptotic regime: omega * dtau << 1 with omega^2 ~ (1+phi^2)/s_eta^2 + 1/s_u^2
    dts = np.array([0.01, 0.005, 0.0025, 0.00125])
    errs = []
    for dt in dts:
        h1, p1 = oracle.leapfrog(h0, p0, s.y, s.lnrv, TH, int(round(L / dt)), dt)
        errs.append(abs(oracle.delta_H(h0, p0, h1, p1, s.y, s.lnrv, TH)))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 1.9 < slope < 2.1


def test_leapfrog_with_mass_reversible_and_second_order():
    T = 300
    s = _series(T, seed=6)
    rng = np.random.default_rng(10)
    minv = rng.uniform(0.5, 2.0, T)
    p0 = rng.standard_normal(T) / np.sqrt(minv)
    h1, p1 = oracle.leapfrog(s.h_true, p0, s.y, s.lnrv, TH, 30, 0.01, minv=minv)
    h2, p2 = oracle.leapfrog(h1, -p1, s.y, s.lnrv, TH, 30, 0.01, minv=minv)
    assert np.max(np.abs(h2 - s.h_true)) < 1e-12
    errs = []
    dts = [0.005, 0.0025, 0.00125]
    for dt in dts:
        h1, p1 = oracle.leapfrog(s.h_true, p0, s.y, s.lnrv, TH, int(round(0.2 / dt)), dt, minv=minv)
        errs.append(abs(oracle.delta_H(s.h_true, p0, h1, p1, s.y, s.lnrv, TH, minv=minv)))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 1.85 < slope < 2.15


def test_leapfrog_free_particle_closed_form():
    """With the force switched off (s_u^2, s_eta^2 huge, y = 0 except the
    constant 1/2) p decreases linearly and h follows the exact parabola:
    leapfrog is exact for a constant force."""
    T = 5
    th = (0.0, 0.0, 0.0, 1e300, 1e300)
    h0 = np.linspace(-1, 1, T)
    p0 = np.linspace(0.5, -0.5, T)
    n, dt = 7, 0.1
    h1, p1 = oracle.leapfrog(h0, p0, np.zeros(T), np.zeros(T), th, n, dt)
    tau = n * dt
    assert np.allclose(p1, p0 - 0.5 * tau, atol=1e-14)
    assert np.allclose(h1, h0 + p0 * tau - 0.25 * tau ** 2, atol=1e-14)


def test_one_ulp_perturbation_stays_small():
    """A 1-ulp change of the input moves h' by far less than the 1e-12 parity bar."""
    T = 2000
    s = _series(T, seed=0)
    p0 = synth.standard_normals(T, 2)
    h1, _ = oracle.leapfrog(s.h0, p0, s.y, s.lnrv, TH, 50, 0.02)
    hp = np.nextafter(s.h0, np.inf)
    h2, _ = oracle.leapfrog(hp, p0, s.y, s.lnrv, TH, 50, 0.02)
    assert np.max(np.abs(h2 - h1) / np.maximum(1, np.abs(h1))) < 1e-13


# --------------------------------------------------------------------------
# Metropolis (Sec. 3)
# --------------------------------------------------------------------------
def test_metropolis_rule():
    assert oracle.metropolis(-0.1, np.log(0.999)) == 1          # dH < 0 always accepts
    assert oracle.metropolis(1.0, np.log(0.5)) == 0              # e^{-1} = 0.37 < 0.5
    assert oracle.metropolis(1.0, np.log(0.3)) == 1
    assert oracle.metropolis(float("nan"), -50.0) == 0
    assert oracle.metropolis(0.7, -0.7) == 0                     # tie rejects


def test_trajectory_reject_restores_h():
    T = 100
    s = _series(T, seed=2)
    p0 = synth.standard_normals(T, 3)
    hA, pA, dH, acc = oracle.trajectory(s.h0, p0, s.y, s.lnrv, TH, 20, 0.02, log_u=0.0)
    assert acc == (0.0 < -dH)
    hB, _, dHB, accB = oracle.trajectory(s.h0, p0, s.y, s.lnrv, TH, 20, 0.02,
                                         log_u=-dH + 1e-9 if dH < 0 else 1.0)
    assert accB == 0 and np.array_equal(hB, s.h0)
    h1, p1 = oracle.leapfrog(s.h0, p0, s.y, s.lnrv, TH, 20, 0.02)
    assert np.array_equal(pA, p1)
    assert dH == pytest.approx(oracle.delta_H(s.h0, p0, h1, p1, s.y, s.lnrv, TH), abs=1e-15)


@pytest.mark.slow
def test_creutz_identity():
    """<exp(-dH)> = 1 for an exact HMC at equilibrium."""
    T = 200
    s = _series(T, seed=8)
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, n_md=10, dtau=0.05, seed=3, n_traj=300)
    r = oracle.chain(r["h"], s.y, s.lnrv, TH, n_md=10, dtau=0.05, seed=4, n_traj=3000)
    w = np.exp(-r["dH"])
    se = stats.batch_means_mcse(w)
    assert abs(w.mean() - 1.0) < 3.5 * se + 1e-3


# --------------------------------------------------------------------------
# tiny T: posterior moments by quadrature
# --------------------------------------------------------------------------
@pytest.mark.slow
def test_T1_posterior_by_quadrature():
    th = TH
    y = np.array([0.9])
    lnrv = np.array([-0.4])
    g = np.linspace(-8, 6, 200001)
    S = np.array([oracle.action(np.array([v]), y, lnrv, th) for v in g[::50]])
    gg = g[::50]
    w = np.exp(-(S - S.min()))
    m = np.sum(gg * w) / np.sum(w)
    v = np.sum((gg - m) ** 2 * w) / np.sum(w)
    r = oracle.chain(np.array([m]), y, lnrv, th, n_md=8, dtau=0.08, seed=21, n_traj=20000,
                     thin=1)
    x = r["snaps"][:, 0]
    se = stats.batch_means_mcse(x)
    assert abs(x.mean() - m) < 3.5 * se
    sev = stats.batch_means_mcse((x - m) ** 2)
    assert abs(x.var() - v) < 3.5 * sev


# --------------------------------------------------------------------------
# Philox4x64-10 against numpy's implementation; Box-Muller closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((5, 1, 2, 3), (7, 9)),
                                     ((2**64 - 1, 2**63, 12345, 999), (2**64 - 1, 2**40 + 3))])
def test_philox_matches_numpy(ctr, key):
    ours = oracle.philox4x64_10(ctr, key)
    # numpy's Philox increments the 256-bit counter before each block
    c = list(ctr)
    carry = 1
    prev = []
    for w in c:
        v = w - carry
        carry = 1 if v < 0 else 0
        prev.append(v % 2**64)
    bg = np.random.Philox(counter=np.array(prev, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4)
    assert [int(v) for v in ours] == [int(v) for v in ref]


def test_u01_and_box_muller_closed_forms():
    assert oracle.u01(0, 53) == 0.5 * 2.0 ** -53
    assert oracle.u01(2**64 - 1, 53) == 1.0 - 0.5 * 2.0 ** -53
    assert oracle.u01(2**64 - 1, 24) == 1.0 - 0.5 * 2.0 ** -24
    u1 = 0.3
    r = np.sqrt(-2 * np.log(u1))
    z0, z1 = oracle.box_muller(u1, 0.0)
    assert z0 == pytest.approx(r, rel=1e-15) and abs(z1) < 1e-15
    z0, z1 = oracle.box_muller(u1, 0.25)
    assert abs(z0) < 1e-15 and z1 == pytest.approx(r, rel=1e-15)


def test_momenta_are_standard_normal_and_scaled_by_mass():
    T = 200001
    p = oracle.draw_momenta(seed=1, series=0, traj=0, T=T)
    assert abs(p.mean()) < 4 / np.sqrt(T)
    assert abs(p.var() - 1) < 4 * np.sqrt(2 / T)
    from scipy import stats as sps
    assert sps.kstest(p, "norm").pvalue > 1e-3
    minv = np.full(T, 4.0)
    p2 = oracle.draw_momenta(seed=1, series=0, traj=0, T=T, minv=minv)
    assert np.allclose(p2, p / 2.0, rtol=0, atol=0)
    # different trajectory counters give different streams
    p3 = oracle.draw_momenta(seed=1, series=0, traj=1, T=T)
    assert abs(np.corrcoef(p, p3)[0, 1]) < 4 / np.sqrt(T)
    lu = np.array([oracle.draw_log_u(5, 0, k) for k in range(20000)])
    assert abs(np.exp(lu).mean() - 0.5) < 4 * np.sqrt(1 / 12 / 20000)


# --------------------------------------------------------------------------
# theta update: each conditional draw against its closed-form law
# --------------------------------------------------------------------------
def test_gibbs_conditionals_follow_closed_forms():
    T = 400
    s = _series(T, seed=13)
    h = s.h_true
    phi, mu, xi, se2, su2 = TH
    n = 4000
    z_xi, g_u, z_mu, g_eta = [], [], [], []
    for k in range(n):
        th1, _ = oracle.gibbs_theta(h, s.lnrv, TH, seed=100, series=0, traj=k, mask=0b01111)
        xi1, su1, mu1, se1 = th1[2], th1[4], th1[1], th1[3]
        r = s.lnrv - h
        z_xi.append((xi1 - r.mean()) / np.sqrt(su2 / T))
        g_u.append(np.sum((r - xi1) ** 2) / (2 * su1))
        w0, w1 = 1 - phi ** 2, (1 - phi) ** 2
        num = w0 * h[0] + (1 - phi) * np.sum(h[1:] - phi * h[:-1])
        den = w0 + (T - 1) * w1
        z_mu.append((mu1 - num / den) * np.sqrt(den / se2))
        x = h - mu1
        Q = (1 - phi ** 2) * x[0] ** 2 + np.sum((x[1:] - phi * x[:-1]) ** 2)
        g_eta.append(Q / (2 * se1))
    from scipy import stats as sps
    assert sps.kstest(z_xi, "norm").pvalue > 1e-3
    assert sps.kstest(z_mu, "norm").pvalue > 1e-3
    assert sps.kstest(g_u, "gamma", args=(T / 2,)).pvalue > 1e-3
    assert sps.kstest(g_eta, "gamma", args=(T / 2,)).pvalue > 1e-3


def test_gibbs_phi_step_targets_its_conditional():
    """phi-only updates (mu, s_eta^2, h fixed) leave p(phi | .) proportional to
    sqrt(1-phi^2) exp(-Q(phi)/(2 s_eta^2)) on (-1,1) invariant: the chain's
    mean and variance match 1-D quadrature."""
    T = 30
    s = _series(T, seed=14)
    h = s.h_true
    phi0, mu, xi, se2, su2 = TH
    g = np.linspace(-0.999999, 0.999999, 200001)
    x = h - mu
    Q = ((1 - g ** 2) * x[0] ** 2 + ((x[1:, None] - g[None, :] * x[:-1, None]) ** 2).sum(0))
    lw = 0.5 * np.log(1 - g ** 2) - Q / (2 * se2)
    w = np.exp(lw - lw.max())
    m = np.sum(g * w) / np.sum(w)
    v = np.sum((g - m) ** 2 * w) / np.sum(w)
    th = TH
    xs = []
    for k in range(20000):
        th, _ = oracle.gibbs_theta(h, s.lnrv, th, seed=200, series=0, traj=k, mask=0b10000)
        xs.append(th[0])
    xs = np.array(xs)
    se = stats.batch_means_mcse(xs)
    assert abs(xs.mean() - m) < 3.5 * se
    sev = stats.batch_means_mcse((xs - m) ** 2)
    assert abs(xs.var() - v) < 3.5 * sev


# --------------------------------------------------------------------------
# ESS estimator on AR(1) with known integrated autocorrelation time
# --------------------------------------------------------------------------
def test_ess_geyer_on_ar1():
    rng = np.random.default_rng(0)
    n, m = 4000, 64
    for rho in (0.0, 0.5, 0.9):
        x = np.empty((n, m))
        x[0] = rng.standard_normal(m) / np.sqrt(1 - rho ** 2)
        for t in range(1, n):
            x[t] = rho * x[t - 1] + rng.standard_normal(m)
        tau = (1 + rho) / (1 - rho)
        ess = stats.ess_geyer(x)
        assert abs(np.mean(ess) / (n / tau) - 1) < 0.1


def test_batch_means_mcse_iid():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((10000, 50))
    se = stats.batch_means_mcse(x)
    assert abs(np.mean(se) / (1 / np.sqrt(10000)) - 1) < 0.1
