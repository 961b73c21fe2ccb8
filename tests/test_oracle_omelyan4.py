"""Pins of the oracle's fourth-order integrator (Omelyan, Mryglod and Folk,
Comput. Phys. Commun. 146, 188 (2002): the force-gradient-free scheme with
five drifts and four kicks per step; one of the higher-order integrators Sec. 3
cites)."""
import pathlib
import re

import numpy as np

import oracle
from paper_1603_08114_gb300 import synth

TH = synth.THETA_STD
ROOT = pathlib.Path(__file__).resolve().parents[1]


def _coeffs():
    c = oracle.PEFRL
    xi, lam, chi = c["xi"], c["lambda"], c["chi"]
    a = [xi, chi, 1 - 2 * (chi + xi), chi, xi]
    b = [(1 - 2 * lam) / 2, lam, lam, (1 - 2 * lam) / 2]
    return a, b


def test_constants_agree_and_are_consistent():
    """The C oracle's and the C-ABI header's constants are the Python ones;
    drifts and kicks each sum to one (consistency)."""
    src = (ROOT / "oracle" / "rsv_oracle.c").read_text()
    hdr = (ROOT / "include" / "rsv.h").read_text()
    for name, key in (("XI", "xi"), ("LAMBDA", "lambda"), ("CHI", "chi")):
        m = re.search(r"#define ORC_PEFRL_%s \(?([0-9.eE+-]+)\)?" % name, src)
        assert m and float(m.group(1)) == oracle.PEFRL[key], name
        m = re.search(r"#define RSV_OMELYAN4_%s \(?([0-9.eE+-]+)\)?" % name, hdr)
        assert m and float(m.group(1)) == oracle.PEFRL[key], name
    a, b = _coeffs()
    assert abs(sum(a) - 1) < 1e-15 and abs(sum(b) - 1) < 1e-15


def test_coefficients_are_fourth_order_on_the_harmonic_oscillator():
    """Composed as 2x2 maps for H = p^2/2 + q^2/2 (drift [[1, a h], [0, 1]],
    kick [[1, 0], [-b h, 1]]), one step differs from the exact rotation by
    O(h^5): the local error's log-log slope is 5 (a second-order set of
    coefficients would give 3).  Independent of the oracle's code."""
    a, b = _coeffs()

    def step(h):
        M = np.eye(2)
        for s in range(5):
            M = np.array([[1, a[s] * h], [0, 1]]) @ M
            if s < 4:
                M = np.array([[1, 0], [-b[s] * h, 1]]) @ M
        return M
    hs = np.array([0.2, 0.1, 0.05, 0.025])
    err = [np.abs(step(h) - np.array([[np.cos(h), np.sin(h)], [-np.sin(h), np.cos(h)]])).max()
           for h in hs]
    slope = np.polyfit(np.log(hs), np.log(err), 1)[0]
    assert abs(slope - 5.0) < 0.2, slope


def test_reversible_with_and_without_mass():
    s = synth.rsv_series(2000, TH, seed=0)
    p = synth.standard_normals(2000, 2)
    for minv in (None, np.random.default_rng(3).uniform(0.5, 2.0, 2000)):
        q = p if minv is None else p / np.sqrt(minv)
        h1, p1 = oracle.omelyan4(s.h_true, q, s.y, s.lnrv, TH, 20, 0.04, minv=minv)
        h2, p2 = oracle.omelyan4(h1, -p1, s.y, s.lnrv, TH, 20, 0.04, minv=minv)
        assert np.max(np.abs(h2 - s.h_true)) < 1e-12 and np.max(np.abs(-p2 - q)) < 1e-12


def test_dH_scales_as_dtau_to_the_fourth():
    s = synth.rsv_series(2000, TH, seed=0)
    p = synth.standard_normals(2000, 4)
    dts = [0.08, 0.04, 0.02, 0.01]
    e = []
    for dt in dts:
        n = int(round(0.4 / dt))
        h1, p1 = oracle.omelyan4(s.h_true, p, s.y, s.lnrv, TH, n, dt)
        e.append(abs(oracle.delta_H(s.h_true, p, h1, p1, s.y, s.lnrv, TH)))
    slope = np.polyfit(np.log(dts), np.log(e), 1)[0]
    assert abs(slope - 4.0) < 0.2, slope


def test_beats_second_order_minimum_norm_at_small_steps():
    """At equal force evaluations per trajectory (length 0.4) and small steps
    the fourth-order error is far below the second-order minimum-norm one's."""
    s = synth.rsv_series(2000, TH, seed=0)
    rng = np.random.default_rng(1)
    for dt in (0.025, 0.0125):
        n = int(round(0.4 / dt))
        e4, e2 = [], []
        for _ in range(4):
            p = rng.standard_normal(2000)
            h1, p1 = oracle.omelyan4(s.h_true, p, s.y, s.lnrv, TH, n, dt)
            e4.append(oracle.delta_H(s.h_true, p, h1, p1, s.y, s.lnrv, TH))
            h2, p2 = oracle.omelyan2(s.h_true, p, s.y, s.lnrv, TH, 2 * n, dt / 2)
            e2.append(oracle.delta_H(s.h_true, p, h2, p2, s.y, s.lnrv, TH))
        assert np.sqrt(np.mean(np.square(e4))) < 0.3 * np.sqrt(np.mean(np.square(e2)))


def test_trajectory_and_chain_dispatch_the_integrator():
    s = synth.rsv_series(200, TH, seed=0)
    p = synth.standard_normals(200, 5)
    h1, p1 = oracle.omelyan4(s.h_true, p, s.y, s.lnrv, TH, 10, 0.05)
    dh = oracle.delta_H(s.h_true, p, h1, p1, s.y, s.lnrv, TH)
    ht, pt, dHt, acc = oracle.trajectory(s.h_true, p, s.y, s.lnrv, TH, 10, 0.05, -1e300,
                                         integrator="omelyan4")
    assert acc == 1 and np.array_equal(ht, h1) and np.array_equal(pt, p1) and dHt == dh
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, 10, 0.05, 3, 4, integrator="omelyan4")
    r2 = oracle.chain(s.h_true, s.y, s.lnrv, TH, 10, 0.05, 3, 4, integrator="omelyan2")
    assert not np.array_equal(r["dH"], r2["dH"])
