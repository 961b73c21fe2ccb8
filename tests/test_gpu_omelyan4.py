"""GPU fourth-order minimum-norm integrator (rsv_set_integrator(RSV_OMELYAN4))
against the FP64 oracle: trajectories (FP64 1e-12 / 1e-9, mixed 1e-4 / 1e-3),
tiles with the fourfold halo, a mass (whose kicks of two sizes the mixed path
scales), leverage, chains, batched plans, and the T = 2^20 workload."""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_08114_gb300 import synth

pytestmark = pytest.mark.gpu
TH = synth.THETA_STD


@pytest.fixture(scope="module")
def rsv():
    from paper_1603_08114_gb300 import rsv as r
    return r


@pytest.fixture(scope="module")
def ctx(rsv):
    c = rsv.Context(0)
    yield c
    c.close()


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def rel_h(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def _case(rsv, ctx, T, n_md, dtau, prec, minv=None, schedule=None, seed=0, rho=0.0):
    s = (synth.rsv_series(T, TH, seed=seed) if rho == 0.0
         else synth.rsv_series_leverage(T, TH, rho, seed=seed))
    p0 = synth.standard_normals(T, seed + 100)
    if minv is not None:
        p0 = p0 / np.sqrt(minv.astype(np.float64))
    h, p = dev(s.h_true), dev(p0)
    rsv.rsv_set_integrator(ctx, "omelyan4")
    rsv.rsv_set_leverage(ctx, rho)
    if schedule:
        rsv.rsv_set_schedule(ctx, *schedule)
    try:
        dH, acc = rsv.rsv_hmc_trajectory(ctx, h, p, dev(s.y), dev(s.lnrv), TH, n_md, dtau,
                                         prec=prec,
                                         minv=None if minv is None else dev(minv, torch.float32),
                                         log_u=dev([-1e300]))
        rsv.rsv_sync_status(ctx)
    finally:
        rsv.rsv_set_schedule(ctx)
        rsv.rsv_set_leverage(ctx, 0.0)
        rsv.rsv_set_integrator(ctx, "leapfrog")
    mv = None if minv is None else minv.astype(np.float64)
    th = TH + (rho,)
    h1, p1 = oracle.omelyan4(s.h_true, p0, s.y, s.lnrv, th, n_md, dtau, minv=mv)
    dHr = oracle.delta_H(s.h_true, p0, h1, p1, s.y, s.lnrv, th, minv=mv)
    assert int(acc.item()) == 1
    return rel_h(h.cpu().numpy(), h1), rel_h(p.cpu().numpy(), p1), abs(dH.item() - dHr)


@pytest.mark.parametrize("T", [1, 2, 3, 33, 513, 2000, 65537])
def test_trajectory_fp64_matches_oracle(rsv, ctx, T):
    eh, ep, ed = _case(rsv, ctx, T, 10, 0.08, "fp64")
    assert eh < 1e-12 and ep < 1e-11 and ed < 1e-9, (eh, ep, ed)


@pytest.mark.parametrize("T", [1, 2, 33, 2000, 65537])
def test_trajectory_mixed_matches_oracle(rsv, ctx, T):
    eh, ep, ed = _case(rsv, ctx, T, 10, 0.08, "mixed")
    assert eh < 1e-4 and ep < 1e-3 and ed < 1e-3, (eh, ep, ed)


@pytest.mark.parametrize("prec,sched,tol", [
    ("fp64", (128, 4, 512 - 2 * (4 * 10 + 1) - 3), 1e-12),
    ("mixed", (64, 8, 512 - 2 * (4 * 10 + 1) - 3), 1e-4),
    ("mixed", (608, 12, 608 * 12 - 2 * (4 * 10 + 1) - 3), 1e-4)])
def test_many_tiles_with_the_fourfold_halo(rsv, ctx, prec, sched, tol):
    """Four force evaluations per step: a tile's owned sites are exact only
    with a halo of 4 n_md + 1; forced small tiles, ragged last tile."""
    eh, ep, ed = _case(rsv, ctx, 20011, 10, 0.08, prec, schedule=sched)
    assert eh < tol and ed < (1e-9 if prec == "fp64" else 1e-3), (eh, ed)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_with_mass(rsv, ctx, prec, tol):
    """The mixed path holds -kick/m for the first kick size and scales it for
    the other; the state stays within tolerance of the FP64 oracle."""
    T = 4097
    minv = np.random.default_rng(1).uniform(0.5, 2.0, T).astype(np.float32)
    eh, ep, ed = _case(rsv, ctx, T, 10, 0.06, prec, minv=minv)
    assert eh < tol and ed < (1e-9 if prec == "fp64" else 1e-3), (eh, ed)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_with_leverage(rsv, ctx, prec, tol):
    eh, ep, ed = _case(rsv, ctx, 4097, 10, 0.06, prec, rho=synth.RHO_STD, seed=3)
    assert eh < tol and ed < (1e-9 if prec == "fp64" else 1e-3), (eh, ed)


@pytest.mark.parametrize("prec,tol", [("fp64", (1e-12, 1e-9)), ("mixed", (1e-4, 1e-3))])
def test_full_size_T2p20(rsv, ctx, prec, tol):
    """The single-chain large series at the scheme's benchmark length."""
    eh, ep, ed = _case(rsv, ctx, 1 << 20, 4, 0.125, prec, seed=1)
    assert eh < tol[0] and ed < tol[1], (eh, ed)


def test_chain_fp64_matches_oracle_chain(rsv, ctx):
    T, n, n_md, dtau, seed = 2000, 12, 5, 0.1, 17
    s = synth.rsv_series(T, TH, seed=0)
    h = dev(s.h_true)
    dHg = torch.empty(n, dtype=torch.float64, device="cuda")
    accg = torch.empty(n, dtype=torch.int32, device="cuda")
    rsv.rsv_set_integrator(ctx, "omelyan4")
    try:
        rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), dev(TH), n_md, dtau, n, seed=seed,
                          dH_out=dHg, accept_out=accg)
        rsv.rsv_sync_status(ctx)
    finally:
        rsv.rsv_set_integrator(ctx, "leapfrog")
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, n_md, dtau, seed, n, integrator="omelyan4")
    assert np.array_equal(accg.cpu().numpy(), r["accept"])
    assert np.max(np.abs(dHg.cpu().numpy() - r["dH"])) < 1e-9
    assert rel_h(h.cpu().numpy(), r["h"]) < 1e-11


def test_batched_plan_keeps_its_integrator(rsv, ctx):
    Ts = [7, 700, 3000, 9000]
    off = np.concatenate([[0], np.cumsum(Ts)]).astype(np.int64)
    ys, ls, hs = [], [], []
    for i, T in enumerate(Ts):
        s = synth.rsv_series(T, TH, seed=50 + i)
        ys.append(s.y)
        ls.append(s.lnrv)
        hs.append(s.h_true)
    y, lr, ht = np.concatenate(ys), np.concatenate(ls), np.concatenate(hs)
    th = np.tile(np.asarray(TH), (len(Ts), 1))
    p0 = np.random.default_rng(3).standard_normal(off[-1])
    rsv.rsv_set_integrator(ctx, "omelyan4")
    rsv.rsv_set_schedule(ctx, 128, 4, 512 - 2 * (4 * 8 + 1) - 3)
    try:
        plan = rsv.Plan(ctx, off, 8, "mixed")
    finally:
        rsv.rsv_set_schedule(ctx)
        rsv.rsv_set_integrator(ctx, "leapfrog")
    assert plan.info()["split_series"] > 0
    h, p = dev(ht), dev(p0)
    dH = torch.empty(len(Ts), dtype=torch.float64, device="cuda")
    rsv.rsv_hmc_batched(ctx, plan, h, dev(y), dev(lr), dev(th.ravel()), 0.06, p=p,
                        log_u=dev(np.full(len(Ts), -1e300)), dH_out=dH)
    rsv.rsv_sync_status(ctx)
    h, dH = h.cpu().numpy(), dH.cpu().numpy()
    for i in range(len(Ts)):
        a, b = off[i], off[i + 1]
        h1, p1 = oracle.omelyan4(ht[a:b], p0[a:b], y[a:b], lr[a:b], TH, 8, 0.06)
        assert rel_h(h[a:b], h1) < 1e-4
        assert abs(dH[i] - oracle.delta_H(ht[a:b], p0[a:b], h1, p1, y[a:b], lr[a:b], TH)) < 1e-3
    plan.close()
