"""GPU RSV model with leverage (rsv_set_leverage) against the FP64 oracle:
S(h) and dS/dh, trajectories (FP64 1e-12 / 1e-9, mixed 1e-4 / 1e-3) of
both integrators, tiles, a mass, chains, batched plans, the 2^20-site
workload, the refusals of the theta update, and rho = 0 restoring eqs. (1)-(3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_08114_gb300 import synth

pytestmark = pytest.mark.gpu
TH = synth.THETA_STD
RHO = synth.RHO_STD


@pytest.fixture(scope="module")
def rsv():
    from paper_1603_08114_gb300 import rsv as r
    return r


@pytest.fixture(scope="module")
def ctx(rsv):
    c = rsv.Context(0)
    yield c
    c.close()


@pytest.fixture
def lev(rsv, ctx):
    """Leverage on for one test; always switched off afterwards."""
    def on(rho=RHO):
        rsv.rsv_set_leverage(ctx, rho)
    yield on
    rsv.rsv_set_leverage(ctx, 0.0)
    rsv.rsv_set_schedule(ctx)
    rsv.rsv_set_integrator(ctx, "leapfrog")


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def rel_h(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


@pytest.mark.parametrize("rho", [-0.6, 0.4])
@pytest.mark.parametrize("T", [1, 2, 3, 1000, 100003])
def test_action_and_force_match_oracle(rsv, ctx, lev, T, rho):
    s = synth.rsv_series_leverage(T, TH, rho, seed=T)
    h = s.h_true + 0.2 * np.random.default_rng(1).standard_normal(T)
    lev(rho)
    S = rsv.rsv_action(ctx, dev(h), dev(s.y), dev(s.lnrv), TH)
    F = rsv.rsv_force(ctx, dev(h), dev(s.y), dev(s.lnrv), TH)
    rsv.rsv_sync_status(ctx)
    Sr = oracle.action(h, s.y, s.lnrv, TH + (rho,))
    Fr = oracle.force(h, s.y, s.lnrv, TH + (rho,))
    assert abs(S.item() - Sr) <= 1e-12 * max(1.0, abs(Sr)) * max(1.0, np.sqrt(T))
    assert rel_h(F.cpu().numpy(), Fr) < 1e-12


def _case(rsv, ctx, lev, T, n_md, dtau, prec, rho=RHO, integrator="leapfrog", minv=None,
          schedule=None, seed=0):
    s = synth.rsv_series_leverage(T, TH, rho, seed=seed)
    p0 = synth.standard_normals(T, seed + 100)
    if minv is not None:
        p0 = p0 / np.sqrt(minv.astype(np.float64))
    h, p = dev(s.h_true), dev(p0)
    lev(rho)
    rsv.rsv_set_integrator(ctx, integrator)
    if schedule:
        rsv.rsv_set_schedule(ctx, *schedule)
    dH, acc = rsv.rsv_hmc_trajectory(ctx, h, p, dev(s.y), dev(s.lnrv), TH, n_md, dtau, prec=prec,
                                     minv=None if minv is None else dev(minv, torch.float32),
                                     log_u=dev([-1e300]))
    rsv.rsv_sync_status(ctx)
    mv = None if minv is None else minv.astype(np.float64)
    th = TH + (rho,)
    if integrator == "leapfrog":
        h1, p1 = oracle.leapfrog(s.h_true, p0, s.y, s.lnrv, th, n_md, dtau, minv=mv)
    else:
        h1, p1 = oracle.omelyan2(s.h_true, p0, s.y, s.lnrv, th, n_md, dtau, minv=mv)
    dHr = oracle.delta_H(s.h_true, p0, h1, p1, s.y, s.lnrv, th, minv=mv)
    assert int(acc.item()) == 1
    return rel_h(h.cpu().numpy(), h1), rel_h(p.cpu().numpy(), p1), abs(dH.item() - dHr)


@pytest.mark.parametrize("T", [1, 2, 3, 33, 513, 2000, 65537])
def test_trajectory_fp64_matches_oracle(rsv, ctx, lev, T):
    eh, ep, ed = _case(rsv, ctx, lev, T, 40, 0.02, "fp64")
    assert eh < 1e-12 and ep < 1e-11 and ed < 1e-9, (eh, ep, ed)


@pytest.mark.parametrize("T", [1, 2, 3, 33, 513, 2000, 65537])
def test_trajectory_mixed_matches_oracle(rsv, ctx, lev, T):
    eh, ep, ed = _case(rsv, ctx, lev, T, 40, 0.02, "mixed")
    assert eh < 1e-4 and ep < 1e-3 and ed < 1e-3, (eh, ep, ed)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
@pytest.mark.parametrize("rho", [-0.9, 0.7])
def test_strong_leverage_and_the_minimum_norm_integrator(rsv, ctx, lev, prec, tol, rho):
    eh, ep, ed = _case(rsv, ctx, lev, 4099, 12, 0.05, prec, rho=rho, integrator="omelyan2")
    assert eh < tol and ed < (1e-9 if prec == "fp64" else 1e-3), (eh, ed)


@pytest.mark.parametrize("prec,sched,tol", [
    ("fp64", (128, 4, 512 - 2 * (30 + 1) - 3), 1e-12),
    ("fp64", (64, 8, 512 - 2 * (30 + 1) - 3), 1e-12),
    ("mixed", (64, 8, 512 - 2 * (30 + 1) - 3), 1e-4),
    ("mixed", (608, 12, 608 * 12 - 2 * (30 + 1) - 3), 1e-4),
    ("mixed", (256, 20, 256 * 20 - 2 * (30 + 1) - 3), 1e-4)])
def test_many_tiles(rsv, ctx, lev, prec, sched, tol):
    """Forced small tiles with a ragged last tile: the leverage term reaches
    one site to the left (w_{t-1}), inside the halo of n_md + 1."""
    eh, ep, ed = _case(rsv, ctx, lev, 20011, 30, 0.02, prec, schedule=sched)
    assert eh < tol and ed < (1e-9 if prec == "fp64" else 1e-3), (eh, ed)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_with_mass(rsv, ctx, lev, prec, tol):
    T = 4097
    minv = np.random.default_rng(1).uniform(0.5, 2.0, T).astype(np.float32)
    eh, ep, ed = _case(rsv, ctx, lev, T, 20, 0.03, prec, minv=minv)
    assert eh < tol and ed < (1e-9 if prec == "fp64" else 1e-3), (eh, ed)


def test_full_size_T2p20_mixed(rsv, ctx, lev):
    """2^20 sites, 100 x 0.005 in the launch configuration of the single-chain
    workload, mixed precision, every site against the oracle."""
    eh, ep, ed = _case(rsv, ctx, lev, 1 << 20, 100, 0.005, "mixed", seed=1)
    assert eh < 1e-4 and ed < 1e-3, (eh, ed)


def test_chain_fp64_matches_oracle_chain(rsv, ctx, lev):
    T, n, n_md, dtau, seed = 2000, 20, 25, 0.03, 13
    s = synth.rsv_series_leverage(T, TH, RHO, seed=0)
    h = dev(s.h_true)
    dHg = torch.empty(n, dtype=torch.float64, device="cuda")
    accg = torch.empty(n, dtype=torch.int32, device="cuda")
    lev()
    rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), dev(TH), n_md, dtau, n, seed=seed,
                      dH_out=dHg, accept_out=accg)
    rsv.rsv_sync_status(ctx)
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH + (RHO,), n_md, dtau, seed, n)
    assert np.array_equal(accg.cpu().numpy(), r["accept"])
    assert np.max(np.abs(dHg.cpu().numpy() - r["dH"])) < 1e-9
    assert rel_h(h.cpu().numpy(), r["h"]) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_batched_plan(rsv, ctx, lev, prec, tol):
    Ts = [1, 7, 700, 3000, 9000]
    off = np.concatenate([[0], np.cumsum(Ts)]).astype(np.int64)
    ys, ls, hs, ths = [], [], [], []
    rng = np.random.default_rng(3)
    for i, T in enumerate(Ts):
        th = (rng.uniform(0.85, 0.98), rng.normal(-0.5, 0.3), -0.2, rng.uniform(0.02, 0.1), 0.1)
        s = synth.rsv_series_leverage(T, th, RHO, seed=40 + i)
        ys.append(s.y)
        ls.append(s.lnrv)
        hs.append(s.h_true)
        ths.append(th)
    y, lr, ht = np.concatenate(ys), np.concatenate(ls), np.concatenate(hs)
    p0 = np.random.default_rng(2).standard_normal(off[-1])
    lev()
    rsv.rsv_set_schedule(ctx, 128, 4, 512 - 2 * (15 + 1) - 3)
    plan = rsv.Plan(ctx, off, 15, prec)
    rsv.rsv_set_schedule(ctx)
    assert plan.info()["split_series"] > 0
    h, p = dev(ht), dev(p0)
    dH = torch.empty(len(Ts), dtype=torch.float64, device="cuda")
    rsv.rsv_hmc_batched(ctx, plan, h, dev(y), dev(lr), dev(np.asarray(ths).ravel()), 0.04, p=p,
                        log_u=dev(np.full(len(Ts), -1e300)), dH_out=dH)
    rsv.rsv_sync_status(ctx)
    h, dH = h.cpu().numpy(), dH.cpu().numpy()
    for i in range(len(Ts)):
        a, b = off[i], off[i + 1]
        th = tuple(ths[i]) + (RHO,)
        h1, p1 = oracle.leapfrog(ht[a:b], p0[a:b], y[a:b], lr[a:b], th, 15, 0.04)
        assert rel_h(h[a:b], h1) < tol
        dHr = oracle.delta_H(ht[a:b], p0[a:b], h1, p1, y[a:b], lr[a:b], th)
        assert abs(dH[i] - dHr) < (1e-9 if prec == "fp64" else 1e-3)
    # a plan keeps its leverage setting: running it without leverage is refused
    rsv.rsv_set_leverage(ctx, 0.0)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_batched(ctx, plan, dev(ht), dev(y), dev(lr), dev(np.asarray(ths).ravel()),
                            0.04)
    plan.close()


def test_theta_update_refused_and_bad_rho(rsv, ctx, lev):
    T = 100
    s = synth.rsv_series_leverage(T, TH, RHO, seed=0)
    lev()
    th = dev(TH)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_gibbs_theta(ctx, dev(s.h_true), dev(s.lnrv), th, seed=1)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_chain(ctx, dev(s.h_true), dev(s.y), dev(s.lnrv), th, 10, 0.02, 2,
                          update_theta=True)
    for bad in (1.0, -1.0, float("nan")):
        with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
            rsv.rsv_set_leverage(ctx, bad)
    assert np.array_equal(th.cpu().numpy(), np.asarray(TH))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rho_zero_restores_the_plain_model(rsv, ctx, lev, prec):
    """Switching leverage on and back off gives bit for bit the trajectory of a
    context that never had it."""
    T = 3000
    s = synth.rsv_series(T, TH, seed=4)
    p0 = synth.standard_normals(T, 8)
    outs = []
    for rho in (None, 0.0):
        if rho is not None:
            lev(-0.5)
            rsv.rsv_hmc_trajectory(ctx, dev(s.h_true), dev(p0), dev(s.y), dev(s.lnrv), TH, 10,
                                   0.02, prec=prec)
            lev(rho)
        h = dev(s.h_true)
        dH, _ = rsv.rsv_hmc_trajectory(ctx, h, dev(p0), dev(s.y), dev(s.lnrv), TH, 30, 0.02,
                                       prec=prec, log_u=dev([-1e300]))
        rsv.rsv_sync_status(ctx)
        outs.append((h.cpu().numpy(), dH.item()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_block_that_does_not_fit_is_refused(rsv, ctx, lev):
    """Leverage and a mass add two per-site arrays to shared memory: a forced
    block of 512 x 16 sites no longer fits on an SM and the call returns
    RSV_EINVAL before any launch (the automatic planner skips such shapes)."""
    T = 20000
    s = synth.rsv_series_leverage(T, TH, RHO, seed=2)
    minv = dev(np.ones(T), torch.float32)
    lev()
    rsv.rsv_set_schedule(ctx, 512, 16, 512 * 16 - 2 * 11 - 3)
    h = dev(s.h_true)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_trajectory(ctx, h, None, dev(s.y), dev(s.lnrv), TH, 10, 0.02,
                               prec="mixed", minv=minv)
    rsv.rsv_set_schedule(ctx)
    rsv.rsv_hmc_trajectory(ctx, h, None, dev(s.y), dev(s.lnrv), TH, 10, 0.02, prec="mixed",
                           minv=minv)
    rsv.rsv_sync_status(ctx)
