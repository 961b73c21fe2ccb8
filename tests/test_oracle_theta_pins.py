"""Pins of the oracle's theta update against 1-D quadrature of the model (CPU).

The paper does not describe its theta update (Sec. 2 uses the code of its ref.
[Takaishi4]); the oracle draws each component of theta from its full
conditional under flat priors on phi, mu, xi and 1/sigma^2 priors on both
variances.  Here each conditional is NOT restated from the oracle's closed
forms: the unnormalised log conditional of one component is the log of the
joint density of eqs. (1)-(3) (the lnRV equation and the AR(1) law of h with
the stationary law of h_1), written factor by factor with scipy's normal
log-density, plus the log prior, evaluated on a dense grid with the other
components and h held fixed.  Its mean and variance by quadrature must match
those of 10^4 independent oracle draws within 3.5 Monte-Carlo standard errors.

The mutant tests compile copies of the oracle with one plausible mistake each
(a shape T/2 -> (T-1)/2, a dropped stationary term,
(T-1)(1-phi)^2 -> T(1-phi)^2 in mu's precision, ...) and check that the
quadrature pin rejects every one of them, so the pins are not vacuous.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from scipy import stats as sps

import oracle
from paper_1603_08114_gb300 import synth

# component index in theta = (phi, mu, xi, s_eta^2, s_u^2) and its mask bit
COMP = {"xi": (2, 1), "sig_u2": (4, 2), "mu": (1, 4), "sig_eta2": (3, 8)}
N_DRAWS = 10000

# Settings: small T makes the T-dependence of each conditional visible; the
# variance conditionals need a shape well above 4 for a finite fourth moment
# of the draws (T = 20 gives 10); the last setting is the benchmark's theta.
SETTINGS = {
    "T8_phi0.3": (8, (0.3, -0.5, -0.2, 0.05, 0.1), 31),
    "T20_phi0.4": (20, (0.4, -0.5, -0.2, 0.05, 0.1), 32),
    "T200_std": (200, synth.THETA_STD, 33),
}
CASES = [("xi", "T8_phi0.3"), ("mu", "T8_phi0.3"), ("sig_u2", "T20_phi0.4"),
         ("sig_eta2", "T20_phi0.4")] + [(c, "T200_std") for c in COMP]


def log_joint(h, lnrv, phi, mu, xi, se2, su2):
    """ln p(h, lnRV | theta) + ln prior(theta) from eqs. (2)-(3) and the
    stationary law of h_1, one normal factor per site.  Each parameter may be
    an array (a grid); the result broadcasts over it."""
    phi, mu, xi, se2, su2 = (np.asarray(v, dtype=np.float64)[..., None]
                             for v in (phi, mu, xi, se2, su2))
    rv = sps.norm.logpdf(lnrv[None, :], loc=xi + h[None, :], scale=np.sqrt(su2)).sum(-1)
    h1 = sps.norm.logpdf(h[0], loc=mu[..., 0], scale=np.sqrt(se2[..., 0] / (1 - phi[..., 0] ** 2)))
    ar = sps.norm.logpdf(h[None, 1:], loc=mu + phi * (h[None, :-1] - mu),
                         scale=np.sqrt(se2)).sum(-1)
    prior = -np.log(se2[..., 0]) - np.log(su2[..., 0])
    return rv + h1 + ar + prior


def quadrature_moments(logp_of, lo, hi, log_axis=False, n=40001):
    """Mean and variance of the density exp(logp) on (lo, hi): a coarse grid
    finds where the mass is, a fine grid there integrates it.  With log_axis
    the grid is uniform in ln(value) (the Jacobian is included)."""
    def on(a, b):
        u = np.linspace(a, b, n)
        v = np.exp(u) if log_axis else u
        lp = logp_of(v) + (u if log_axis else 0.0)
        return u, v, lp
    a, b = (np.log(lo), np.log(hi)) if log_axis else (lo, hi)
    for _ in range(3):  # zoom onto the region within e^-60 of the maximum
        u, v, lp = on(a, b)
        keep = np.nonzero(lp > lp.max() - 60.0)[0]
        i0, i1 = max(keep[0] - 1, 0), min(keep[-1] + 1, n - 1)
        a, b = u[i0], u[i1]
    u, v, lp = on(a, b)
    assert lp[0] < lp.max() - 40 and lp[-1] < lp.max() - 40, "grid does not cover the mass"
    w = np.exp(lp - lp.max())
    m = np.sum(v * w) / np.sum(w)
    var = np.sum((v - m) ** 2 * w) / np.sum(w)
    return m, var


def conditional_moments(name, h, lnrv, th):
    idx, _ = COMP[name]

    def logp(v):
        args = list(th)
        args[idx] = v
        return log_joint(h, lnrv, *args)
    if name in ("xi", "mu"):
        return quadrature_moments(logp, -20.0, 20.0)
    return quadrature_moments(logp, 1e-6, 1e3, log_axis=True)


def oracle_draws(gibbs, name, h, lnrv, th, seed):
    idx, bit = COMP[name]
    out = np.empty(N_DRAWS)
    for k in range(N_DRAWS):
        t = gibbs(h, lnrv, th, seed, k, bit)
        out[k] = t[idx]
        # the other components are untouched by a one-component sweep
        assert all(t[i] == th[i] for i in range(5) if i != idx)
    return out


def _oracle_gibbs(h, lnrv, th, seed, traj, mask):
    return oracle.gibbs_theta(h, lnrv, th, seed=seed, series=0, traj=traj, mask=mask)[0]


def check_against_quadrature(gibbs, name, setting):
    """(ok, z_mean, z_var): the draws' mean and variance against quadrature,
    in units of their Monte-Carlo standard errors (independent draws)."""
    T, th, seed = SETTINGS[setting]
    s = synth.rsv_series(T, th, seed=seed)
    m, v = conditional_moments(name, s.h_true, s.lnrv, th)
    x = oracle_draws(gibbs, name, s.h_true, s.lnrv, th, seed=500 + seed)
    se_m = x.std() / np.sqrt(len(x))
    dev2 = (x - m) ** 2
    se_v = dev2.std() / np.sqrt(len(x))
    z_m = (x.mean() - m) / se_m
    z_v = (dev2.mean() - v) / se_v
    return abs(z_m) < 3.5 and abs(z_v) < 3.5, z_m, z_v


def test_log_joint_matches_the_model_written_out():
    """The quadrature's density is the model's: at one theta it equals the
    normal log-densities of eqs. (2)-(3) written out by hand (2 pi terms
    included), and its h-dependent part is minus the oracle's action S(h) up
    to the y-terms of eq. (1), which do not involve these components."""
    T = 7
    th = (0.6, -0.4, -0.1, 0.07, 0.12)
    s = synth.rsv_series(T, th, seed=3)
    phi, mu, xi, se2, su2 = th
    h, lr = s.h_true, s.lnrv
    by_hand = (-0.5 * T * np.log(2 * np.pi * su2) - np.sum((lr - xi - h) ** 2) / (2 * su2)
               - 0.5 * np.log(2 * np.pi * se2 / (1 - phi ** 2))
               - (1 - phi ** 2) * (h[0] - mu) ** 2 / (2 * se2)
               - 0.5 * (T - 1) * np.log(2 * np.pi * se2)
               - np.sum((h[1:] - mu - phi * (h[:-1] - mu)) ** 2) / (2 * se2)
               - np.log(se2) - np.log(su2))
    assert float(log_joint(h, lr, *th)[0]) == pytest.approx(by_hand, rel=1e-13)
    # h-dependence: differences between two states equal minus the oracle's
    # action differences once the y-terms h/2 + y^2/2 e^{-h} are removed
    h2 = h + 0.1 * np.sin(np.arange(T))
    d_joint = float((log_joint(h2, lr, *th) - log_joint(h, lr, *th))[0])
    y0 = np.zeros(T)
    d_S = oracle.action(h2, y0, lr, th) - oracle.action(h, y0, lr, th)
    d_y = np.sum(h2 / 2 - h / 2)  # the h/2 of the y-terms with y = 0
    assert d_joint == pytest.approx(-(d_S - d_y), rel=1e-11)


@pytest.mark.parametrize("name,setting", CASES)
def test_theta_conditional_matches_quadrature(name, setting):
    ok, z_m, z_v = check_against_quadrature(_oracle_gibbs, name, setting)
    assert ok, (name, setting, z_m, z_v)


# ---------------------------------------------------------------------------
# Mutants: one plausible mistake each, planted in a copy of the oracle's C
# source (never in the oracle itself), must fail the quadrature pin.
# ---------------------------------------------------------------------------
MUTANTS = {
    # mu: the AR terms counted T times instead of T - 1 (precision and mean)
    "mu_precision_T": ("(Td - 1.0) * w1", "Td * w1", "mu", "T8_phi0.3"),
    # mu: the stationary weight 1 - phi^2 of h_1 dropped from the mean
    "mu_stationary_mean": ("sum_add(&num, w0 * h[0]);", "sum_add(&num, h[0]);", "mu",
                           "T8_phi0.3"),
    # xi: variance s_u^2 / (T - 1)
    "xi_variance": ("sqrt(th->sig_u2 / Td)", "sqrt(th->sig_u2 / (Td - 1.0))", "xi",
                    "T8_phi0.3"),
    # s_u^2: inverse-gamma shape (T - 1)/2
    "su2_shape": ("double g = stream_gamma(&st, 0.5 * Td);",
                  "double g = stream_gamma(&st, 0.5 * (Td - 1.0));", "sig_u2", "T20_phi0.4"),
    # s_eta^2: the stationary term (1 - phi^2) x_1^2 left out of Q
    "seta2_no_stationary": ("sum_add(&q, (1.0 - phi * phi) * x0 * x0);", "(void)x0;",
                            "sig_eta2", "T20_phi0.4"),
    # s_eta^2: inverse-gamma shape (T - 1)/2
    "seta2_shape": ("double g2 = stream_gamma(&st, 0.5 * Td);",
                    "double g2 = stream_gamma(&st, 0.5 * (Td - 1.0));", "sig_eta2",
                    "T20_phi0.4"),
}


def _mutant_gibbs(tmp_path, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rsv_oracle.c")).read()
    assert old in src, old
    mutated = src.replace(old, new)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(c), "-lm"])
    L = ctypes.CDLL(str(so))
    D = ctypes.POINTER(ctypes.c_double)
    L.orc_gibbs_theta.restype = ctypes.c_int
    L.orc_gibbs_theta.argtypes = [D, D, ctypes.c_long, ctypes.POINTER(oracle.Theta),
                                  ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]

    def gibbs(h, lnrv, th, seed, traj, mask):
        h = np.ascontiguousarray(h, dtype=np.float64)
        lnrv = np.ascontiguousarray(lnrv, dtype=np.float64)
        t = oracle.Theta(*[float(v) for v in th])
        L.orc_gibbs_theta(h.ctypes.data_as(D), lnrv.ctypes.data_as(D), len(h),
                          ctypes.byref(t), int(seed), 0, int(traj), int(mask))
        return t.as_tuple()
    return gibbs


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_quadrature_pin_rejects_planted_mistake(tmp_path, mutant):
    old, new, name, setting = MUTANTS[mutant]
    gibbs = _mutant_gibbs(tmp_path, old, new)
    ok, z_m, z_v = check_against_quadrature(gibbs, name, setting)
    assert not ok, (mutant, z_m, z_v)
