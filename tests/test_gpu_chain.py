"""The persistent chain (one cooperative launch for a whole rsv_hmc_chain call
of a mixed single series) against the per-trajectory launches: the same
states, theta records, dH, decisions and snapshots bit for bit; and its
bounded grid-barrier wait, which reports RSV_ETIMEOUT when it runs out.
Both paths are checked against the FP64 oracle elsewhere (the persistent one
is the default, so every mixed chain test runs it)."""
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


def run(rsv, ctx, s, persistent, n, n_md, dtau, minv=None, update_theta=True, thin=1, fb=0,
        seed=5, integrator="leapfrog"):
    """One chain call; both paths on the tiling the persistent chain takes
    (the planner prefers another block shape for per-trajectory launches, and
    results depend on the tiling through their rounding only)."""
    T = len(s.y)
    rsv.rsv_set_integrator(ctx, integrator)
    cs = rsv.rsv_chain_schedule(ctx, T, n_md, "mixed", with_mass=minv is not None)
    rsv.rsv_set_schedule(ctx, cs["threads"], cs["sites_per_thread"], cs["tile"])
    h, th = dev(s.h_true), dev(TH)
    snaps = torch.full((n // thin, T), float("nan"), dtype=torch.float32, device="cuda")
    ths = torch.full((n, 5), float("nan"), dtype=torch.float64, device="cuda")
    dH = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    acc = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    used = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rsv.rsv_set_persistent(ctx, persistent)
    rsv.rsv_set_integrator(ctx, integrator)
    try:
        rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), th, n_md, dtau, n, prec="mixed",
                          minv=minv, seed=seed, traj0=3, update_theta=update_theta, snaps=snaps,
                          thin=thin, theta_out=ths, dH_out=dH, accept_out=acc,
                          fallback_window=fb, mass_used_out=used)
        # a trajectory whose dH is not finite is a rejection (the fallback
        # case's steps are that large)
        rsv.rsv_sync_status(ctx, allow_nonfinite=True)
    finally:
        rsv.rsv_set_persistent(ctx, True)
        rsv.rsv_set_integrator(ctx, "leapfrog")
        rsv.rsv_set_schedule(ctx)
    return {k: v.cpu().numpy() for k, v in dict(h=h, th=th, snaps=snaps, ths=ths, dH=dH,
                                                 acc=acc, used=used).items()}


def same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("T", [3000, 1 << 17, 1 << 20])
@pytest.mark.parametrize("mass", [False, True])
def test_persistent_chain_equals_per_trajectory_launches(rsv, ctx, T, mass):
    """A whole series (one block) and series cut into tiles (19 and 147
    blocks), with and without a mass, theta sampled, every state recorded."""
    s = synth.rsv_series(T, TH, seed=7)
    minv = None
    n_md, dtau = 20, 0.02
    if mass:
        minv = dev(1.0 / (25.0 + 10.0 * np.exp(synth.log_uniforms(T, 8))), torch.float32)
        dtau = 0.1
    a = run(rsv, ctx, s, True, 12, n_md, dtau, minv=minv)
    b = run(rsv, ctx, s, False, 12, n_md, dtau, minv=minv)
    same(a, b)
    assert 0 < a["acc"].sum() < 12 or a["acc"].sum() == 12


def test_persistent_chain_thinned_fixed_theta_and_fallback(rsv, ctx):
    """thin = 3 over 8 trajectories (the last due snapshot after the loop),
    theta fixed (its records are the given theta), and a mass whose step is
    too large, so that the fallback window switches it off part-way."""
    T = 1 << 17
    s = synth.rsv_series(T, TH, seed=9)
    minv = dev(np.full(T, 1.0 / 30.0), torch.float32)
    for ut in (False, True):
        a = run(rsv, ctx, s, True, 8, 10, 0.02, update_theta=ut, thin=3)
        b = run(rsv, ctx, s, False, 8, 10, 0.02, update_theta=ut, thin=3)
        same(a, b)
    a = run(rsv, ctx, s, True, 9, 10, 0.5, minv=minv, fb=3)
    b = run(rsv, ctx, s, False, 9, 10, 0.5, minv=minv, fb=3)
    same(a, b)
    assert a["used"][0] == 0   # the mass was switched off


@pytest.mark.parametrize("integrator", ["omelyan2", "omelyan4"])
def test_persistent_chain_other_integrators(rsv, ctx, integrator):
    s = synth.rsv_series(1 << 17, TH, seed=11)
    a = run(rsv, ctx, s, True, 6, 4, 0.1, integrator=integrator)
    b = run(rsv, ctx, s, False, 6, 4, 0.1, integrator=integrator)
    same(a, b)


def test_barrier_wait_that_runs_out_reports_timeout(rsv, ctx):
    """A one-cycle wait limit: the first block to reach the grid barrier gives
    up before the others arrive; every block stops, the status word reports
    RSV_ETIMEOUT, and the context runs the next chain normally."""
    T = 1 << 17
    s = synth.rsv_series(T, TH, seed=13)
    rsv.rsv_set_wait_limit(ctx, 1)
    try:
        h, th = dev(s.h_true), dev(TH)
        rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), th, 10, 0.02, 4, prec="mixed", seed=1,
                          update_theta=True)
        with pytest.raises(rsv.RSVError, match="RSV_ETIMEOUT"):
            rsv.rsv_sync_status(ctx)
    finally:
        rsv.rsv_set_wait_limit(ctx, 0)
    a = run(rsv, ctx, s, True, 4, 10, 0.02)
    b = run(rsv, ctx, s, False, 4, 10, 0.02)
    same(a, b)


def test_wait_limit_rejects_negative(rsv, ctx):
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_set_wait_limit(ctx, -1)


def test_planner_block_shapes_at_the_measured_sizes(rsv, ctx):
    """The planner's choices where they were measured: the headline chain
    (T = 2^20, mass, 78 steps) runs persistent on 384 x 20 (140 tiles; per
    trajectory 88.5 us against 92.1 on 448 x 16), and a series of 2^22 sites
    cut into 4 waves of tiles takes the same full blocks (0.382 ms a
    trajectory against 0.449 on 288 x 20).  A fixed schedule is reported
    with its own tile."""
    cs = rsv.rsv_chain_schedule(ctx, 1 << 20, 78, "mixed", with_mass=True)
    assert (cs["threads"], cs["sites_per_thread"], cs["persistent"]) == (384, 20, True)
    assert cs["tile"] == 384 * 20 - 2 * 79 - 3
    cs = rsv.rsv_chain_schedule(ctx, 1 << 22, 100, "mixed", with_mass=False)
    assert (cs["threads"], cs["sites_per_thread"], cs["persistent"]) == (384, 20, False)
    rsv.rsv_set_schedule(ctx, 384, 20, 7000)
    try:
        cs = rsv.rsv_chain_schedule(ctx, 1 << 20, 78, "mixed", with_mass=True)
        assert cs["tile"] == 7000
    finally:
        rsv.rsv_set_schedule(ctx)
