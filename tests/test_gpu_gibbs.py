"""GPU theta update and theta-sampling chains against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import stats
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


@pytest.mark.parametrize("T", [1, 2, 3, 100, 2000, 65537])
@pytest.mark.parametrize("mask", [31, 0b10000, 0b01111])
def test_gibbs_sweep_matches_oracle(rsv, ctx, T, mask):
    s = synth.rsv_series(T, TH, seed=T)
    h = s.h_true + 0.05 * synth.standard_normals(T, 1)
    for traj in range(4):
        th = dev(TH)
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        rsv.rsv_gibbs_theta(ctx, dev(h), dev(s.lnrv), th, seed=5, series=0, traj=traj, mask=mask,
                            phi_acc_out=acc)
        ref, racc = oracle.gibbs_theta(h, s.lnrv, TH, seed=5, series=0, traj=traj, mask=mask)
        got = th.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-13), (got, ref)
        assert int(acc.item()) == racc


def test_chain_with_theta_fp64_matches_oracle(rsv, ctx):
    T, n, n_md, dtau, seed = 2000, 25, 50, 0.02, 21
    s = synth.rsv_series(T, TH, seed=0)
    h = dev(s.h_true)
    th = dev(TH)
    ths = torch.empty(n, 5, dtype=torch.float64, device="cuda")
    acc = torch.empty(n, dtype=torch.int32, device="cuda")
    rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), th, n_md, dtau, n, seed=seed,
                      update_theta=True, theta_out=ths, accept_out=acc)
    rsv.rsv_sync_status(ctx)
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, n_md, dtau, seed, n, update_theta=True)
    assert np.array_equal(acc.cpu().numpy(), r["accept"])
    assert np.allclose(ths.cpu().numpy(), r["thetas"], rtol=1e-9, atol=1e-11)
    assert np.max(np.abs(h.cpu().numpy() - r["h"])) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_chain_theta_posterior_means_agree_with_oracle(rsv, ctx, prec):
    """The 2000-site workload with theta sampled (50 x 0.02 per trajectory).
    Posterior means of theta and of a few h_t from the GPU chain lie within
    3.5 combined Monte-Carlo standard errors (sd / sqrt(ESS), Geyer) of the
    oracle chain's (different Philox seed, so the chains are independent).
    theta mixes slowly (phi, s_eta^2 autocorrelation times of ~100), hence
    4000 trajectories."""
    T, n, n_md, dtau, burn = 2000, 4000, 50, 0.02, 500
    s = synth.rsv_series(T, TH, seed=0)
    # start from a posterior-typical state: at h = lnRV - xi the RV residuals
    # vanish and the first s_u^2 draw is degenerate
    h = dev(s.h_true)
    th = dev(TH)
    ths = torch.empty(n, 5, dtype=torch.float64, device="cuda")
    snaps = torch.empty(n // 2, T, dtype=torch.float32, device="cuda")
    rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), th, n_md, dtau, n, prec=prec, seed=31,
                      update_theta=True, theta_out=ths, snaps=snaps, thin=2)
    rsv.rsv_sync_status(ctx)
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, n_md, dtau, 32, n, update_theta=True, thin=2)
    def mcse(x):
        return x.std(0, ddof=1) / np.sqrt(stats.ess_geyer(x))

    g = ths.cpu().numpy()[burn:]
    o = r["thetas"][burn:]
    z = np.abs(g.mean(0) - o.mean(0)) / np.sqrt(mcse(g) ** 2 + mcse(o) ** 2)
    assert np.all(z < 3.5), z
    cols = [0, 7, 500, 1999]
    gh = snaps.cpu().numpy()[burn // 2:, cols].astype(np.float64)
    oh = r["snaps"][burn // 2:, cols]
    z = np.abs(gh.mean(0) - oh.mean(0)) / np.sqrt(mcse(gh) ** 2 + mcse(oh) ** 2)
    assert np.all(z < 3.5), z


@pytest.mark.parametrize("T", [1, 2, 3, 100, 2000, 65537])
def test_gibbs_sweep_mixed_close_to_oracle(rsv, ctx, T):
    """The mixed sweep (double-float statistics, FP32 draws from 23-bit uniforms
    of the same stream positions) against the FP64 oracle's sweep from the
    same 23-bit uniforms: every variate agrees to FP32-level distance (1e-4
    relative), unless one of the sweep's accept/reject decisions lies within
    1e-4 of its boundary in the oracle (its smallest decision margin), where
    FP32 rounding may take the other branch.  theta comes out FP32-valued."""
    s = synth.rsv_series(T, TH, seed=T)
    h = s.h_true + 0.05 * synth.standard_normals(T, 1)
    for traj in range(8):
        th = dev(TH)
        rsv.rsv_gibbs_theta(ctx, dev(h), dev(s.lnrv), th, seed=5, series=0, traj=traj,
                            prec="mixed")
        got = th.cpu().numpy()
        ref, _, margin = oracle.gibbs_theta_margin(h, s.lnrv, TH, seed=5, series=0, traj=traj,
                                                   bits=23)
        assert np.array_equal(got.astype(np.float32).astype(np.float64), got)
        rel = np.abs(got - np.array(ref)) / np.abs(np.array(ref))
        assert rel.max() <= 1e-4 or margin < 1e-4, (traj, rel, margin)
