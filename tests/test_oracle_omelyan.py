"""Pins of the oracle's minimum-norm integrator (Omelyan, Mryglod, Folk 2002;
one of the higher-order integrators Sec. 3 cites)."""
import numpy as np

import oracle
from paper_1603_08114_gb300 import synth

TH = synth.THETA_STD


def _series(T=2000, seed=0):
    return synth.rsv_series(T, TH, seed=seed)


def test_lambda_is_the_minimum_norm_root():
    """lambda = 1/2 - c/12 + 1/(6c), c = (2 sqrt(326) + 36)^(1/3), the root of the
    error-norm minimisation, agrees with the oracle's constant and the C header's."""
    c = (2.0 * np.sqrt(326.0) + 36.0) ** (1.0 / 3.0)
    lam = 0.5 - c / 12.0 + 1.0 / (6.0 * c)
    assert abs(lam - oracle.LAMBDA_2MN) < 1e-15
    import re
    import pathlib
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "rsv.h").read_text()
    m = re.search(r"#define RSV_OMELYAN2_LAMBDA ([0-9.eE+-]+)", hdr)
    assert m and abs(float(m.group(1)) - lam) < 1e-15


def test_half_lambda_is_the_leapfrog():
    """lambda = 1/2: drift dtau/2, two kicks of dtau/2 at the same point, drift
    dtau/2 -- eqs. (6)-(8) with the force step split in two."""
    s = _series()
    p = synth.standard_normals(2000, 1)
    a = oracle.leapfrog(s.h_true, p, s.y, s.lnrv, TH, 30, 0.01)
    b = oracle.omelyan2(s.h_true, p, s.y, s.lnrv, TH, 30, 0.01, lam=0.5)
    assert np.max(np.abs(a[0] - b[0])) < 1e-13 and np.max(np.abs(a[1] - b[1])) < 1e-12


def test_reversible_with_and_without_mass():
    s = _series()
    p = synth.standard_normals(2000, 2)
    for minv in (None, np.random.default_rng(3).uniform(0.5, 2.0, 2000)):
        q = p if minv is None else p / np.sqrt(minv)
        h1, p1 = oracle.omelyan2(s.h_true, q, s.y, s.lnrv, TH, 40, 0.02, minv=minv)
        h2, p2 = oracle.omelyan2(h1, -p1, s.y, s.lnrv, TH, 40, 0.02, minv=minv)
        assert np.max(np.abs(h2 - s.h_true)) < 1e-12 and np.max(np.abs(-p2 - q)) < 1e-12


def test_dH_scales_as_dtau_squared():
    s = _series()
    p = synth.standard_normals(2000, 4)
    dts = [0.04, 0.02, 0.01, 0.005]
    e = []
    for dt in dts:
        n = int(round(0.4 / dt))
        h1, p1 = oracle.omelyan2(s.h_true, p, s.y, s.lnrv, TH, n, dt)
        e.append(abs(oracle.delta_H(s.h_true, p, h1, p1, s.y, s.lnrv, TH)))
    slope = np.polyfit(np.log(dts), np.log(e), 1)[0]
    assert abs(slope - 2.0) < 0.15, slope


def test_smaller_energy_error_than_leapfrog_at_equal_force_evaluations():
    """At the same number of force evaluations per trajectory (length 0.5),
    the minimum-norm integrator's rms dH is an order of magnitude below the
    leapfrog's on this posterior (measured ~25x)."""
    s = _series()
    rng = np.random.default_rng(0)
    for nf in (40, 80):
        lf, mn = [], []
        for _ in range(6):
            p = rng.standard_normal(2000)
            h1, p1 = oracle.leapfrog(s.h_true, p, s.y, s.lnrv, TH, nf, 0.5 / nf)
            lf.append(oracle.delta_H(s.h_true, p, h1, p1, s.y, s.lnrv, TH))
            h2, p2 = oracle.omelyan2(s.h_true, p, s.y, s.lnrv, TH, nf // 2, 0.5 / (nf // 2))
            mn.append(oracle.delta_H(s.h_true, p, h2, p2, s.y, s.lnrv, TH))
        assert np.sqrt(np.mean(np.square(mn))) < 0.1 * np.sqrt(np.mean(np.square(lf)))


def test_trajectory_and_chain_dispatch_the_integrator():
    s = _series(200)
    p = synth.standard_normals(200, 5)
    h1, p1 = oracle.omelyan2(s.h_true, p, s.y, s.lnrv, TH, 10, 0.05)
    dh = oracle.delta_H(s.h_true, p, h1, p1, s.y, s.lnrv, TH)
    ht, pt, dHt, acc = oracle.trajectory(s.h_true, p, s.y, s.lnrv, TH, 10, 0.05, -1e300,
                                         integrator="omelyan2")
    assert acc == 1 and np.array_equal(ht, h1) and np.array_equal(pt, p1) and dHt == dh
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, 10, 0.05, 3, 4, integrator="omelyan2")
    r0 = oracle.chain(s.h_true, s.y, s.lnrv, TH, 10, 0.05, 3, 4)
    assert not np.array_equal(r["dH"], r0["dH"])
