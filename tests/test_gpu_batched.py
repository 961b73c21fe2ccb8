"""Many independent series in one persistent launch, against the FP64 oracle per series."""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_08114_gb300 import synth

pytestmark = pytest.mark.gpu


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
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))) if len(a) else 0.0


def make_batch(Ts, seed=0):
    rng = np.random.default_rng(seed)
    n = len(Ts)
    th = np.stack([rng.uniform(0.85, 0.99, n), rng.normal(-0.5, 0.3, n), rng.normal(-0.2, 0.1, n),
                   rng.uniform(0.02, 0.1, n), rng.uniform(0.05, 0.2, n)], axis=1)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(Ts)
    y, lr, ht = [], [], []
    for s in range(n):
        ser = synth.rsv_series(int(Ts[s]), tuple(th[s]), seed=1000 + s)
        y.append(ser.y)
        lr.append(ser.lnrv)
        ht.append(ser.h_true)
    return off, th, np.concatenate(y), np.concatenate(lr), np.concatenate(ht)


TS_MIX = [1, 2, 3, 33, 64, 500, 513, 1000, 2000, 31, 4097, 9000, 700, 8192, 1, 250]


@pytest.mark.parametrize("prec,tol_h,tol_dh,gap", [("fp64", 1e-12, 1e-9, 1e-9),
                                                   ("mixed", 1e-4, 1e-3, 1e-2)])
@pytest.mark.parametrize("sched", [None, (64, 8, 200)])
def test_batched_trajectory_matches_oracle_per_series(rsv, ctx, prec, tol_h, tol_dh, gap, sched):
    n_md, dtau = 20, 0.02
    off, th, y, lr, ht = make_batch(TS_MIX)
    n = len(TS_MIX)
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(off[-1])
    lu = np.log(rng.random(n))
    lu[::3] = -1e300  # always accept: compare h'
    if sched:
        rsv.rsv_set_schedule(ctx, *sched)
    try:
        plan = rsv.Plan(ctx, off, n_md, prec)
    finally:
        rsv.rsv_set_schedule(ctx)
    info = plan.info()
    if sched:
        assert info["split_series"] > 0
    h = dev(ht)
    p = dev(p0)
    dH = torch.empty(n, dtype=torch.float64, device="cuda")
    acc = torch.empty(n, dtype=torch.int32, device="cuda")
    rsv.rsv_hmc_batched(ctx, plan, h, dev(y), dev(lr), dev(th.ravel()), dtau, p=p, log_u=dev(lu),
                        dH_out=dH, accept_out=acc)
    rsv.rsv_sync_status(ctx)
    h, p, dH, acc = h.cpu().numpy(), p.cpu().numpy(), dH.cpu().numpy(), acc.cpu().numpy()
    for s in range(n):
        a, b = off[s], off[s + 1]
        h1, p1 = oracle.leapfrog(ht[a:b], p0[a:b], y[a:b], lr[a:b], th[s], n_md, dtau)
        dHr = oracle.delta_H(ht[a:b], p0[a:b], h1, p1, y[a:b], lr[a:b], th[s])
        assert abs(dH[s] - dHr) <= tol_dh, (s, dH[s], dHr)
        if abs(dHr + lu[s]) > gap:
            assert acc[s] == oracle.metropolis(dHr, lu[s]), s
        assert rel_h(p[a:b], p1) <= 10 * tol_h, s
        if acc[s]:
            assert rel_h(h[a:b], h1) <= tol_h, s
        else:
            assert np.array_equal(h[a:b], ht[a:b]), s
    plan.close()


def test_batched_chain_fp64_matches_oracle_chains(rsv, ctx):
    """Several trajectories with Philox draws per series (counter word 3 = series)."""
    n_md, dtau, n_traj, seed = 20, 0.02, 6, 77
    Ts = [5, 700, 2000, 9000, 64]
    off, th, y, lr, ht = make_batch(Ts, seed=1)
    n = len(Ts)
    plan = rsv.Plan(ctx, off, n_md, "fp64")
    h = dev(ht)
    dH = torch.empty(n_traj * n, dtype=torch.float64, device="cuda")
    acc = torch.empty(n_traj * n, dtype=torch.int32, device="cuda")
    rsv.rsv_hmc_batched(ctx, plan, h, dev(y), dev(lr), dev(th.ravel()), dtau, seed=seed,
                        traj0=3, n_traj=n_traj, dH_out=dH, accept_out=acc)
    rsv.rsv_sync_status(ctx)
    h = h.cpu().numpy()
    dH = dH.cpu().numpy().reshape(n_traj, n)
    acc = acc.cpu().numpy().reshape(n_traj, n)
    for s in range(n):
        a, b = off[s], off[s + 1]
        r = oracle.chain(ht[a:b], y[a:b], lr[a:b], th[s], n_md, dtau, seed, n_traj, traj0=3,
                         series=s)
        assert np.array_equal(acc[:, s], r["accept"]), s
        assert np.max(np.abs(dH[:, s] - r["dH"])) < 1e-9, s
        assert rel_h(h[a:b], r["h"]) < 1e-11, s
    plan.close()


def test_batched_workload_plan_and_graph_replay(rsv, ctx):
    """The 4096-series workload (T ~ U{500..8192}, theta per series): plan shape,
    a CUDA-graph replay equal to the eager call, finite dH everywhere."""
    b = synth.rsv_batch(4096, 500, 8192, seed=2)
    n = 4096
    plan = rsv.Plan(ctx, b.offsets, 50, "mixed")
    info = plan.info()
    assert info["bins"] >= 1 and info["grid"] >= 1
    rsv.rsv_reserve(ctx, int(b.offsets[-1]), n)
    y, lr, th = dev(b.y), dev(b.lnrv), dev(b.theta.ravel())
    h_e = dev(b.h_true)
    dH_e = torch.empty(n, dtype=torch.float64, device="cuda")
    acc_e = torch.empty(n, dtype=torch.int32, device="cuda")
    rsv.rsv_hmc_batched(ctx, plan, h_e, y, lr, th, 0.02, seed=5, traj0=0, dH_out=dH_e,
                        accept_out=acc_e)
    torch.cuda.synchronize()
    h_g = dev(b.h_true)
    dH_g = torch.empty(n, dtype=torch.float64, device="cuda")
    acc_g = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            rsv.rsv_hmc_batched(ctx, plan, h_g, y, lr, th, 0.02, seed=5, traj0=0, dH_out=dH_g,
                                accept_out=acc_g)
    g.replay()
    torch.cuda.synchronize()
    rsv.rsv_sync_status(ctx)
    assert torch.equal(dH_e, dH_g) and torch.equal(acc_e, acc_g) and torch.equal(h_e, h_g)
    assert torch.isfinite(dH_e).all()
    assert 0.3 < acc_e.float().mean().item() <= 1.0
    plan.close()
