"""Oracle parity at the benchmark's own sampler settings, T = 2^20 sites.

The benchmark runs the mixed path with a trained diagonal mass at 78 x 0.035
(the step its tuner picks), the second-order minimum-norm integrator at
6 x 0.0833 (identity) and 6 x 0.46 (learned mass), and every chain of the
tests elsewhere starts from the generator's latent path.  Here each of those
settings is checked against the FP64 oracle on the same seeded inputs:
FP64 path 1e-12 relative on h' and 1e-9 absolute on dH; mixed path 1e-4 and
1e-3, with identical accept decisions wherever |dH + ln u| > 1e-2 (the
trajectory's drawn uniform and a forced accept, so that h' is compared too).
The mass is trained by the library's own pipeline (plain-sampler moments,
Adam on the BF16 network, clamped inverse mass) on a short run, so it has the
learned mass's shape (nearly constant, m ~ 30, larger at the ends).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_08114_gb300 import synth

pytestmark = pytest.mark.gpu
TH = synth.THETA_STD
T = 1 << 20


@pytest.fixture(scope="module")
def rsv():
    from paper_1603_08114_gb300 import rsv as r
    return r


@pytest.fixture(scope="module")
def ctx(rsv):
    c = rsv.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def series():
    return synth.rsv_series(T, TH, seed=1)


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def rel_h(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


@pytest.fixture(scope="module")
def learned_minv(rsv, ctx, series):
    """An inverse mass from the library's training pipeline (short run)."""
    from paper_1603_08114_gb300 import learned
    s = series
    y, lr = dev(s.y), dev(s.lnrv)
    h = dev(s.h_true)
    th = dev(TH)
    mean, m2, cnt = learned.collect_moments(ctx, h, y, lr, th, 200, 100, 0.005, seed=5)
    tm = learned.train_mass(ctx, y, lr, TH, mean, m2, cnt, steps=300, batch=4096, seed=7)
    minv = tm.minv.cpu().numpy().astype(np.float32)
    m = 1.0 / minv.astype(np.float64)
    assert np.all(np.isfinite(m)) and 10 < np.median(m) < 100
    return minv


def run_case(rsv, ctx, s, h0, n_md, dtau, prec, minv=None, integrator="leapfrog", seed=0,
             force_accept=False):
    p0 = synth.standard_normals(T, seed + 100)
    if minv is not None:
        p0 = p0 / np.sqrt(minv.astype(np.float64))     # p ~ N(0, m)
    log_u = -1e300 if force_accept else float(synth.log_uniforms(1, seed + 200)[0])
    h, p = dev(h0), dev(p0)
    if integrator != "leapfrog":
        rsv.rsv_set_integrator(ctx, integrator)
    try:
        dH, acc = rsv.rsv_hmc_trajectory(ctx, h, p, dev(s.y), dev(s.lnrv), TH, n_md, dtau,
                                         prec=prec,
                                         minv=None if minv is None else dev(minv, torch.float32),
                                         log_u=dev([log_u]))
        rsv.rsv_sync_status(ctx)
    finally:
        rsv.rsv_set_integrator(ctx, "leapfrog")
    mv = None if minv is None else minv.astype(np.float64)
    h1r, p1r, dHr, accr = oracle.trajectory(h0, p0, s.y, s.lnrv, TH, n_md, dtau, log_u, minv=mv,
                                            integrator=integrator)
    return dict(h=h.cpu().numpy(), p=p.cpu().numpy(), dH=dH.item(), acc=int(acc.item()),
                h0=h0, h1r=h1r, p1r=p1r, dHr=dHr, accr=accr, log_u=log_u)


def check(r, tol_h, tol_dh, tol_gap):
    assert abs(r["dH"] - r["dHr"]) <= tol_dh, (r["dH"], r["dHr"])
    if abs(r["dHr"] + r["log_u"]) > tol_gap:
        assert r["acc"] == r["accr"], (r["dHr"], r["log_u"])
    assert rel_h(r["p"], r["p1r"]) <= tol_h * 10
    if r["acc"] and r["accr"]:
        assert rel_h(r["h"], r["h1r"]) <= tol_h
    elif not r["acc"]:
        assert np.array_equal(r["h"], r["h0"])


@pytest.mark.parametrize("force_accept", [True, False])
def test_learned_mass_78x0035_mixed(rsv, ctx, series, learned_minv, force_accept):
    """The headline arm: mixed path, trained mass, 78 x 0.035."""
    r = run_case(rsv, ctx, series, series.h_true, 78, 0.035, "mixed", minv=learned_minv, seed=3,
                 force_accept=force_accept)
    check(r, 1e-4, 1e-3, 1e-2)


def test_learned_mass_78x0035_fp64(rsv, ctx, series, learned_minv):
    r = run_case(rsv, ctx, series, series.h_true, 78, 0.035, "fp64", minv=learned_minv, seed=4,
                 force_accept=True)
    check(r, 1e-12, 1e-9, 1e-9)


@pytest.mark.parametrize("prec,tol", [("fp64", (1e-12, 1e-9, 1e-9)), ("mixed", (1e-4, 1e-3, 1e-2))])
@pytest.mark.parametrize("force_accept", [True, False])
def test_omelyan2_6x0083_identity(rsv, ctx, series, prec, tol, force_accept):
    """The minimum-norm arm with the identity mass: 6 steps of 0.5 / 6."""
    r = run_case(rsv, ctx, series, series.h_true, 6, 0.5 / 6, prec, integrator="omelyan2",
                 seed=5, force_accept=force_accept)
    check(r, *tol)


def test_omelyan2_6x046_learned_mass_mixed(rsv, ctx, series, learned_minv):
    """The minimum-norm arm with the learned mass at its tuned 6 x 0.46."""
    r = run_case(rsv, ctx, series, series.h_true, 6, 0.46, "mixed", minv=learned_minv,
                 integrator="omelyan2", seed=6, force_accept=True)
    check(r, 1e-4, 1e-3, 1e-2)


@pytest.mark.parametrize("n_md,dtau", [(20, 0.0005), (20, 0.001)])
@pytest.mark.parametrize("force_accept", [True, False])
def test_mixed_from_lnrv_minus_xi(rsv, ctx, series, n_md, dtau, force_accept):
    """The chain start h = lnRV - xi (far from the posterior: every site's RV
    residual is zero and the AR terms are large), at steps small enough to be
    accepted from there (the oracle's dH is 0.05 and 0.8)."""
    s = series
    r = run_case(rsv, ctx, s, s.h0, n_md, dtau, "mixed", seed=8, force_accept=force_accept)
    check(r, 1e-4, 1e-3, 1e-2)
