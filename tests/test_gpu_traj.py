"""GPU (C-ABI) against the FP64 oracle: S(h), dS/dh, momenta, trajectories, chains.

Tolerances: FP64 path 1e-12 relative on h' (max |dh| / max(1, |h|)) and 1e-9
absolute on dH; mixed path 1e-4 and 1e-3, with identical accept decisions
wherever |dH + ln u| > 1e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_08114_gb300 import synth

pytestmark = pytest.mark.gpu
TH = synth.THETA_STD
SIZES = [1, 2, 3, 31, 32, 33, 511, 512, 513, 2000, 65537]


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


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T", SIZES)
def test_force_matches_oracle(rsv, ctx, T):
    s = synth.rsv_series(T, TH, seed=T)
    h = s.h_true + 0.2 * synth.standard_normals(T, 3)
    F = rsv.rsv_force(ctx, dev(h), dev(s.y), dev(s.lnrv), TH).cpu().numpy()
    ref = oracle.force(h, s.y, s.lnrv, TH)
    assert np.max(np.abs(F - ref) / np.maximum(1.0, np.abs(ref))) < 1e-13


@pytest.mark.parametrize("T", SIZES + [1 << 20])
def test_action_matches_oracle(rsv, ctx, T):
    s = synth.rsv_series(T, TH, seed=T + 1)
    S = rsv.rsv_action(ctx, dev(s.h0), dev(s.y), dev(s.lnrv), TH).item()
    ref = oracle.action(s.h0, s.y, s.lnrv, TH)
    assert abs(S - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("bits", [53, 23])
def test_momenta_match_oracle_generator(rsv, ctx, bits):
    T = 10001
    minv = np.random.default_rng(4).uniform(0.5, 2.0, T).astype(np.float32)
    for mv in (None, minv):
        p = rsv.rsv_draw_momenta(ctx, 12345, 3, 77, T, None if mv is None else dev(mv, torch.float32),
                                 bits=bits).cpu().numpy()
        ref = oracle.draw_momenta(12345, 3, 77, T, None if mv is None else mv.astype(np.float64),
                                  bits=bits)
        tol = 1e-13 if bits == 53 else 2e-6
        assert np.max(np.abs(p - ref) / np.maximum(1.0, np.abs(ref))) < tol


# ---------------------------------------------------------------------------
def _traj_case(rsv, ctx, T, n_md, dtau, prec, start="h0", minv=None, log_u=None, schedule=None,
               seed=0):
    s = synth.rsv_series(T, TH, seed=seed)
    h0 = s.h0 if start == "h0" else s.h_true
    p0 = synth.standard_normals(T, seed + 100)
    if minv is not None:
        p0 = p0 / np.sqrt(minv.astype(np.float64))
    if log_u is None:
        log_u = float(synth.log_uniforms(1, seed + 200)[0])
    h = dev(h0)
    p = dev(p0)
    if schedule:
        rsv.rsv_set_schedule(ctx, *schedule)
    try:
        dH, acc = rsv.rsv_hmc_trajectory(ctx, h, p, dev(s.y), dev(s.lnrv), TH, n_md, dtau,
                                         prec=prec, minv=None if minv is None else dev(minv, torch.float32),
                                         log_u=dev([log_u]))
        rsv.rsv_sync_status(ctx)
    finally:
        if schedule:
            rsv.rsv_set_schedule(ctx)
    mv = None if minv is None else minv.astype(np.float64)
    h1r, p1r = oracle.leapfrog(h0, p0, s.y, s.lnrv, TH, n_md, dtau, minv=mv)
    dHr = oracle.delta_H(h0, p0, h1r, p1r, s.y, s.lnrv, TH, minv=mv)
    accr = oracle.metropolis(dHr, log_u)
    return dict(h=h.cpu().numpy(), p=p.cpu().numpy(), dH=dH.item(), acc=int(acc.item()), h0=h0,
                h1r=h1r, p1r=p1r, dHr=dHr, accr=accr, log_u=log_u)


def _check(r, tol_h, tol_dh, tol_gap):
    assert abs(r["dH"] - r["dHr"]) <= tol_dh, (r["dH"], r["dHr"])
    if abs(r["dHr"] + r["log_u"]) > tol_gap:
        assert r["acc"] == r["accr"]
    assert rel_h(r["p"], r["p1r"]) <= tol_h * 10
    if r["acc"]:
        assert rel_h(r["h"], r["h1r"]) <= tol_h
    else:
        assert np.array_equal(r["h"], r["h0"])


@pytest.mark.parametrize("T", SIZES)
def test_trajectory_fp64_matches_oracle(rsv, ctx, T):
    r = _traj_case(rsv, ctx, T, 50, 0.02, "fp64", log_u=-1e300)   # always accept: compare h'
    assert r["acc"] == 1
    _check(r, 1e-12, 1e-9, 1e-9)
    r = _traj_case(rsv, ctx, T, 50, 0.02, "fp64", seed=7)
    _check(r, 1e-12, 1e-9, 1e-9)


@pytest.mark.parametrize("T,sched", [(513, (128, 4, 512 - 2 * 21 - 3)),
                                     (2000, (64, 8, 512 - 2 * 21 - 3)),
                                     (65537, (128, 8, 1024 - 2 * 21 - 3)),
                                     (65537, (256, 28, 256 * 28 - 2 * 21 - 3))])
def test_trajectory_fp64_many_tiles(rsv, ctx, T, sched):
    """Forced small tiles: many windows, halos and a ragged last tile."""
    r = _traj_case(rsv, ctx, T, 20, 0.02, "fp64", log_u=-1e300, schedule=sched)
    _check(r, 1e-12, 1e-9, 1e-9)


@pytest.mark.parametrize("T", [1, 33, 2000, 65537])
def test_trajectory_fp64_with_mass(rsv, ctx, T):
    minv = np.random.default_rng(T).uniform(0.5, 2.0, T).astype(np.float32)
    r = _traj_case(rsv, ctx, T, 30, 0.01, "fp64", minv=minv, log_u=-1e300)
    _check(r, 1e-12, 1e-9, 1e-9)


def test_trajectory_drawn_momenta_and_uniform(rsv, ctx):
    T, n_md, dtau, seed, traj = 2000, 50, 0.02, 99, 5
    s = synth.rsv_series(T, TH, seed=0)
    h = dev(s.h0)
    dH, acc = rsv.rsv_hmc_trajectory(ctx, h, None, dev(s.y), dev(s.lnrv), TH, n_md, dtau,
                                     seed=seed, traj=traj)
    p0 = oracle.draw_momenta(seed, 0, traj, T)
    lu = oracle.draw_log_u(seed, 0, traj)
    h1, p1, dHr, accr = oracle.trajectory(s.h0, p0, s.y, s.lnrv, TH, n_md, dtau, lu)
    assert abs(dH.item() - dHr) < 1e-9
    assert int(acc.item()) == accr
    assert rel_h(h.cpu().numpy(), h1) < 1e-12


@pytest.mark.parametrize("T", [1, 2, 33, 513, 2000, 65537])
def test_trajectory_mixed_matches_oracle(rsv, ctx, T):
    r = _traj_case(rsv, ctx, T, 50, 0.02, "mixed", start="h_true", log_u=-1e300)
    _check(r, 1e-4, 1e-3, 1e-2)
    r = _traj_case(rsv, ctx, T, 50, 0.02, "mixed", start="h_true", seed=3)
    _check(r, 1e-4, 1e-3, 1e-2)


@pytest.mark.parametrize("T,sched", [(2000, (64, 8, 512 - 2 * 21 - 3)),
                                     (65537, (384, 20, 384 * 20 - 2 * 21 - 3))])
def test_trajectory_mixed_many_tiles(rsv, ctx, T, sched):
    r = _traj_case(rsv, ctx, T, 20, 0.02, "mixed", start="h_true", log_u=-1e300, schedule=sched)
    _check(r, 1e-4, 1e-3, 1e-2)


def test_trajectory_mixed_with_mass(rsv, ctx):
    T = 4097
    minv = np.random.default_rng(1).uniform(0.5, 2.0, T).astype(np.float32)
    r = _traj_case(rsv, ctx, T, 30, 0.01, "mixed", start="h_true", minv=minv, log_u=-1e300)
    _check(r, 1e-4, 1e-3, 1e-2)


# ---------------------------------------------------------------------------
def test_chain_fp64_matches_oracle_chain(rsv, ctx):
    """C1 shape: T = 2000, 50 x 0.02, Philox momenta and uniforms, theta fixed."""
    T, n, n_md, dtau, seed = 2000, 30, 50, 0.02, 11
    s = synth.rsv_series(T, TH, seed=0)
    h = dev(s.h0)
    th = dev(TH)
    dHg = torch.empty(n, dtype=torch.float64, device="cuda")
    accg = torch.empty(n, dtype=torch.int32, device="cuda")
    snaps = torch.empty(n // 5, T, dtype=torch.float32, device="cuda")
    rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), th, n_md, dtau, n, seed=seed,
                      dH_out=dHg, accept_out=accg, snaps=snaps, thin=5)
    rsv.rsv_sync_status(ctx)
    r = oracle.chain(s.h0, s.y, s.lnrv, TH, n_md, dtau, seed, n, thin=5)
    assert np.array_equal(accg.cpu().numpy(), r["accept"])
    assert np.max(np.abs(dHg.cpu().numpy() - r["dH"])) < 1e-9
    assert rel_h(h.cpu().numpy(), r["h"]) < 1e-11
    assert np.max(np.abs(snaps.cpu().numpy() - r["snaps"])) < 1e-5


def test_chain_mixed_tracks_oracle(rsv, ctx):
    T, n, n_md, dtau, seed = 2000, 10, 50, 0.02, 12
    s = synth.rsv_series(T, TH, seed=0)
    h = dev(s.h_true)
    dHg = torch.empty(n, dtype=torch.float64, device="cuda")
    accg = torch.empty(n, dtype=torch.int32, device="cuda")
    rsv.rsv_hmc_chain(ctx, h, dev(s.y), dev(s.lnrv), dev(TH), n_md, dtau, n, prec="mixed",
                      seed=seed, dH_out=dHg, accept_out=accg)
    rsv.rsv_sync_status(ctx)
    r = oracle.chain(s.h_true, s.y, s.lnrv, TH, n_md, dtau, seed, n, bits=23)
    lu = np.array([oracle.draw_log_u(seed, 0, k) for k in range(n)])
    dHg = dHg.cpu().numpy()
    accg = accg.cpu().numpy()
    # identical decisions while they are not marginal; the chains stay coupled
    for k in range(n):
        if abs(r["dH"][k] + lu[k]) > 1e-2:
            assert accg[k] == r["accept"][k]
        assert abs(dHg[k] - r["dH"][k]) < 1e-3
    assert rel_h(h.cpu().numpy(), r["h"]) < 1e-4


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol_h,tol_dh,tol_gap", [("fp64", 1e-12, 1e-9, 1e-9),
                                                       ("mixed", 1e-4, 1e-3, 1e-2)])
def test_full_size_T2p20(rsv, ctx, prec, tol_h, tol_dh, tol_gap):
    """2^20 sites, 100 x 0.005 (the single-chain large-series workload)."""
    T = 1 << 20
    s = synth.rsv_series(T, TH, seed=1)
    r = _traj_case(rsv, ctx, T, 100, 0.005, prec, start="h_true", log_u=-1e300, seed=1)
    _check(r, tol_h, tol_dh, tol_gap)


def test_full_size_T2p22_mixed_precision_report(rsv, ctx):
    """2^22 sites, THETA_LARGE, 100 x 0.003: FP32 trajectory vs FP64 oracle."""
    T = 1 << 22
    s = synth.rsv_series(T, synth.THETA_LARGE, seed=3)
    p0 = synth.standard_normals(T, 5)
    lu = float(synth.log_uniforms(1, 6)[0])
    h = dev(s.h_true)
    p = dev(p0)
    dH, acc = rsv.rsv_hmc_trajectory(ctx, h, p, dev(s.y), dev(s.lnrv), synth.THETA_LARGE, 100,
                                     0.003, prec="mixed", log_u=dev([-1e300]))
    rsv.rsv_sync_status(ctx)
    h1r, p1r = oracle.leapfrog(s.h_true, p0, s.y, s.lnrv, synth.THETA_LARGE, 100, 0.003)
    dHr = oracle.delta_H(s.h_true, p0, h1r, p1r, s.y, s.lnrv, synth.THETA_LARGE)
    assert rel_h(h.cpu().numpy(), h1r) < 1e-4
    assert abs(dH.item() - dHr) < 1e-3
    assert (lu < -dH.item()) == (lu < -dHr) or abs(dHr + lu) <= 1e-2


@pytest.mark.parametrize("case", ["T2p22", "T2p20_mass", "T2p20_leverage"])
def test_mixed_dH_evaluation_error(rsv, ctx, case):
    """The mixed dH against the oracle's dH of the kernel's own end state (h',
    p' read back) from its own start (p rounded to FP32 as the kernel takes
    it): the evaluation error alone, without the FP32 trajectory's deviation."""
    T, th, n_md, dtau, rho, minv = 1 << 22, synth.THETA_LARGE, 100, 0.003, 0.0, None
    if case != "T2p22":
        T, th, n_md, dtau = 1 << 20, TH, 100, 0.005
    if case == "T2p20_mass":
        minv = np.random.default_rng(4).uniform(0.5, 2.0, T).astype(np.float32)
        dtau = 0.004
    if case == "T2p20_leverage":
        rho = synth.RHO_STD
        s = synth.rsv_series_leverage(T, th, rho, seed=7)
    else:
        s = synth.rsv_series(T, th, seed=3)
    p0 = synth.standard_normals(T, 5)
    if minv is not None:
        p0 = p0 / np.sqrt(minv.astype(np.float64))
    p0 = p0.astype(np.float32).astype(np.float64)
    h, p = dev(s.h_true), dev(p0)
    rsv.rsv_set_leverage(ctx, rho)
    try:
        dH, _ = rsv.rsv_hmc_trajectory(ctx, h, p, dev(s.y), dev(s.lnrv), th, n_md, dtau,
                                       prec="mixed", log_u=dev([-1e300]),
                                       minv=None if minv is None else dev(minv, torch.float32))
        rsv.rsv_sync_status(ctx)
    finally:
        rsv.rsv_set_leverage(ctx, 0.0)
    mv = None if minv is None else minv.astype(np.float64)
    dHe = oracle.delta_H(s.h_true, p0, h.cpu().numpy(), p.cpu().numpy(), s.y, s.lnrv,
                         th + (rho,), minv=mv)
    err = abs(dH.item() - dHe)
    print(f"mixed dH evaluation error {case}: {err:.3e} (dH = {dHe:.4f})")
    assert err < 1e-4, err


# ---------------------------------------------------------------------------
def test_invalid_arguments_rejected(rsv, ctx):
    T = 10
    s = synth.rsv_series(T, TH, seed=0)
    h, y, lr = dev(s.h0), dev(s.y), dev(s.lnrv)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_trajectory(ctx, h, None, y, lr, (1.0, -0.5, -0.2, 0.05, 0.1), 10, 0.02)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_trajectory(ctx, h, None, y, lr, (0.9, -0.5, -0.2, -0.05, 0.1), 10, 0.02)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_trajectory(ctx, h, None, y, lr, TH, 0, 0.02)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_hmc_trajectory(ctx, h, None, y, lr, TH, 10, -0.02)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        rsv.rsv_force(ctx, h, y, lr, TH, F_out=h)
    with pytest.raises(rsv.RSVError, match="RSV_EINVAL"):
        # T = 10 cut into tiles of 5 needs halos of 301 sites: no window holds them
        rsv.rsv_set_schedule(ctx, 64, 8, 5)
        rsv.rsv_hmc_trajectory(ctx, h, None, y, lr, TH, 300, 0.02)
    rsv.rsv_set_schedule(ctx)
    assert np.array_equal(h.cpu().numpy(), s.h0)


def test_nonfinite_dH_rejects_and_reports(rsv, ctx):
    T = 100
    s = synth.rsv_series(T, TH, seed=0)
    y = s.y.copy()
    y[17] = np.inf
    h = dev(s.h0)
    dH, acc = rsv.rsv_hmc_trajectory(ctx, h, None, dev(y), dev(s.lnrv), TH, 5, 0.02, seed=1)
    with pytest.raises(rsv.RSVError, match="RSV_ENONFINITE"):
        rsv.rsv_sync_status(ctx)
    assert int(acc.item()) == 0
    assert np.array_equal(h.cpu().numpy(), s.h0)
    rsv.rsv_sync_status(ctx)  # cleared
