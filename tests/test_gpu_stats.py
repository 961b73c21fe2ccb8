"""The mixed chain's start energy from stored state statistics (model without
leverage): statistics re-centred after a theta update against statistics taken
afresh at the new theta, on the same trajectory."""
import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("T", [3000, 1 << 17])  # one whole series; tiles of a split series
@pytest.mark.parametrize("mass", [False, True])
def test_recentred_statistics_match_a_fresh_record(rsv, ctx, T, mass):
    s = synth.rsv_series(T, TH, seed=3)
    y, lr = dev(s.y), dev(s.lnrv)
    minv = None
    if mass:
        u = np.exp(synth.log_uniforms(T, 7))
        minv = dev(1.0 / (20.0 + 20.0 * u), torch.float32)
    n_md, dtau, seed = 20, 0.08 if mass else 0.02, 11

    # two trajectories with a theta sweep after each: the second one starts
    # from statistics centred at the first one's theta
    hB, thB = dev(s.h_true), dev(TH)
    dB = torch.empty(2, dtype=torch.float64, device="cuda")
    thsB = torch.empty(2, 5, dtype=torch.float64, device="cuda")
    rsv.rsv_hmc_chain(ctx, hB, y, lr, thB, n_md, dtau, 2, prec="mixed", minv=minv, seed=seed,
                      update_theta=True, dH_out=dB, theta_out=thsB)
    # the first trajectory alone: the state and theta the second one started from
    hA, thA = dev(s.h_true), dev(TH)
    dA = torch.empty(1, dtype=torch.float64, device="cuda")
    rsv.rsv_hmc_chain(ctx, hA, y, lr, thA, n_md, dtau, 1, prec="mixed", minv=minv, seed=seed,
                      update_theta=True, dH_out=dA)
    rsv.rsv_sync_status(ctx)
    assert dA.item() == dB[0].item()
    assert torch.equal(thA, thsB[0])
    shift = (thA - dev(TH)).abs().cpu().numpy()
    assert shift[1] > 0 and shift[2] > 0  # mu and xi moved: the centre shifts
    # the second trajectory again, its statistics taken fresh at that theta
    # (FP32-valued, so the call prepares the sweep's own constants and the
    # trajectory is the same); only the evaluation of dH differs, and every
    # term of the re-centring moves dH by far more than the tolerance at these
    # sizes (T dmu / 2 alone is 10 or more).
    dC = torch.empty(1, dtype=torch.float64, device="cuda")
    rsv.rsv_hmc_chain(ctx, hA, y, lr, thA, n_md, dtau, 1, prec="mixed", minv=minv, seed=seed,
                      traj0=1, dH_out=dC)
    rsv.rsv_sync_status(ctx)
    assert np.isfinite(dC.item())
    assert abs(dC.item() - dB[1].item()) < 1e-6, (dC.item(), dB[1].item())


@pytest.mark.parametrize("T", [1, 2, 3, 100, 2000, 1 << 17])
def test_sweep_from_statistics_close_to_oracle(rsv, ctx, T):
    """One mixed trajectory, then the theta sweep, which takes its sums from
    the statistics of the state the trajectory left (no pass over the sites):
    theta lands within FP32-level distance (1e-4 relative) of the FP64
    oracle's sweep of that state from the same 23-bit uniforms, unless one of
    the sweep's accept/reject decisions lies within 1e-4 of its boundary in
    the oracle, where FP32 rounding may take the other branch.  theta comes
    out FP32-valued."""
    import oracle
    s = synth.rsv_series(T, TH, seed=T)
    for traj in range(8):
        h, th = dev(s.h_true), dev(TH)
        rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), th, 20, 0.02, 1, prec="mixed", seed=5,
                          traj0=traj, update_theta=True)
        rsv.rsv_sync_status(ctx)
        got = th.cpu().numpy()
        ref, _, margin = oracle.gibbs_theta_margin(h.cpu().numpy(), s.lnrv, TH, seed=5, series=0,
                                                   traj=traj, bits=23)
        assert np.array_equal(got.astype(np.float32).astype(np.float64), got)
        rel = (np.abs(got - np.array(ref)) / np.abs(np.array(ref))).max()
        assert rel <= 1e-4 or margin < 1e-4, (traj, rel, margin)


@pytest.mark.parametrize("T,update_theta", [(3000, True), (1 << 17, False), (1 << 17, True)])
def test_mixed_chain_snapshots_are_the_states(rsv, ctx, T, update_theta):
    """A snapshot of the mixed chain is written by the next trajectory's load
    pass (the last one by its own kernel): snapshot k is the state after k
    trajectories, rounded to FP32, bit for bit."""
    s = synth.rsv_series(T, TH, seed=4)
    y, lr = dev(s.y), dev(s.lnrv)
    n = 4
    snaps = torch.empty(n, T, dtype=torch.float32, device="cuda")
    h, th = dev(s.h_true), dev(TH)
    rsv.rsv_hmc_chain(ctx, h, y, lr, th, 10, 0.02, n, prec="mixed", seed=9,
                      update_theta=update_theta, snaps=snaps, thin=1)
    for k in range(1, n + 1):
        hk, thk = dev(s.h_true), dev(TH)
        rsv.rsv_hmc_chain(ctx, hk, y, lr, thk, 10, 0.02, k, prec="mixed", seed=9,
                          update_theta=update_theta)
        rsv.rsv_sync_status(ctx)
        assert torch.equal(snaps[k - 1], hk.float()), k


@pytest.mark.parametrize("n,thin", [(6, 3), (7, 3), (8, 3)])
@pytest.mark.parametrize("T", [3000, 1 << 17])
def test_mixed_chain_thinned_snapshots_are_the_states(rsv, ctx, T, n, thin):
    """Snapshots every thin-th trajectory, n not always a multiple of thin: a
    due snapshot is written by the next trajectory's load pass when there is
    one, the last due one by its own kernel; snapshot k is the state after
    (k + 1) thin trajectories, bit for bit."""
    s = synth.rsv_series(T, TH, seed=5)
    y, lr = dev(s.y), dev(s.lnrv)
    snaps = torch.full((n // thin, T), float("nan"), dtype=torch.float32, device="cuda")
    h, th = dev(s.h_true), dev(TH)
    rsv.rsv_hmc_chain(ctx, h, y, lr, th, 10, 0.02, n, prec="mixed", seed=19,
                      update_theta=True, snaps=snaps, thin=thin)
    for k in range(n // thin):
        hk, thk = dev(s.h_true), dev(TH)
        rsv.rsv_hmc_chain(ctx, hk, y, lr, thk, 10, 0.02, (k + 1) * thin, prec="mixed",
                          seed=19, update_theta=True)
        rsv.rsv_sync_status(ctx)
        assert torch.equal(snaps[k], hk.float()), k


@pytest.mark.parametrize("T", [3000, 1 << 17])
def test_mixed_leverage_chain_snapshots_are_the_states(rsv, ctx, T):
    """The same with leverage (rho = -0.4, theta fixed), whose kernel keeps H
    at both ends per site and writes the deferred snapshot from its own
    instantiation of the load pass."""
    s = synth.rsv_series_leverage(T, TH, synth.RHO_STD, seed=6)
    y, lr = dev(s.y), dev(s.lnrv)
    n, thin = 5, 2
    snaps = torch.full((n // thin, T), float("nan"), dtype=torch.float32, device="cuda")
    rsv.rsv_set_leverage(ctx, synth.RHO_STD)
    try:
        h, th = dev(s.h_true), dev(TH)
        rsv.rsv_hmc_chain(ctx, h, y, lr, th, 10, 0.02, n, prec="mixed", seed=23, snaps=snaps,
                          thin=thin)
        for k in range(n // thin):
            hk, thk = dev(s.h_true), dev(TH)
            rsv.rsv_hmc_chain(ctx, hk, y, lr, thk, 10, 0.02, (k + 1) * thin, prec="mixed",
                              seed=23)
            rsv.rsv_sync_status(ctx)
            assert torch.equal(snaps[k], hk.float()), k
    finally:
        rsv.rsv_set_leverage(ctx, 0.0)
