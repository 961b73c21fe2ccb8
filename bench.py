"""Benchmark of the RSV-model HMC volatility update on GB300.

Workload (the single-chain large-series case): T = 2^20 sites of a synthetic
RSV series (phi, mu, xi, s_eta^2, s_u^2) = (0.95, -0.5, -0.2, 0.05, 0.1), seed 1;
one step = one chain segment of 200 HMC sweeps (momenta, 100 leapfrog steps of
dtau = 0.005, dH, Metropolis, then a Gibbs sweep of theta), run by one
rsv_hmc_chain call that also records every trajectory's h and theta for ESS.  The
chain continues from step to step (the warm-up steps are its burn-in).

Headline sampler: mixed precision with the learned diagonal mass (trained
before timing from 10^4 plain-sampler snapshots; its step size tuned to ~0.8
acceptance at the plain sampler's physical trajectory length; identity-mass
fallback).  Reported: leapfrog site-updates/s (T * n_md * trajectories /
time) and ESS/s of h and theta (Geyer ESS over the whole timed chain / its
time), beside the plain mixed and plain FP64 samplers (identity mass,
100 x 0.005) with a check that the learned and identity chains reach the same
per-site posterior moments, the T = 2000 FP64 workload, the T = 2^22 mixed
workload with its error against the FP64 path, the elementary-step sweep of
the paper's Table 2 (B = 1 ... 2048), the 4096-series batched workload, the
RSV model with leverage and the minimum-norm integrator (identity and learned
mass); the MD-only rate, the end-to-end rate from pinned host buffers, the
trajectory kernel's roofline against FP32 and ex2 peaks measured in the same
run, and the CPU oracle's rate.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T_SITES = 1 << 20
N_MD = 100
DTAU = 0.005
N_TRAJ = 200  # trajectories per step (--traj-per-step changes it for profiling runs)
SEED_DATA = 1
METRIC = "leapfrog site-updates/s & ESS/s at T=2^20, mixed+learned vs FP64 plain, 1 GB300"
UNIT = "site-updates/s"
THETA_NAMES = ("phi", "mu", "xi", "sig_eta2", "sig_u2")
WORKLOAD = ("rsv-hmc single chain T=2^20, theta sampled, 200 trajectories per step; "
            "learned mass (tuned dtau, n_md) vs identity 100 x 0.005")
# The method's algorithmic work per site and leapfrog step (eqs. (6)-(8)):
# two half-step drifts of h (2), the force of eq. (7) -- neighbour sum, the
# (1+phi^2) x and phi (x_{t-1} + x_{t+1}) terms with the RV term folded in, the
# exponent argument and the y^2/2 e^{-h} term (5), the kick of p (1), and
# the two FMAs of a diagonal mass (2): 10 FP operations and one exp.
ALG_OPS_PER_SITE_STEP = 10
# What the mixed kernel issues for the same step: the three-point force (5),
# the compensated kick (4) and the compensated drift (4; the two half drifts
# merged), i.e. 3 operations of compensation beyond the method's 10.
IMPL_OPS_PER_SITE_STEP_MIXED = 13
# dram__bytes_read.sum + dram__bytes_write.sum per trajectory of the headline's
# kernel (the persistent chain kernel: one launch's bytes over its
# trajectories; the inputs stay in L2 between trajectories), from the capture
# summarised in profiles/; valid for the kernel revision it was taken on.
# (the capture: `python bench.py --profile-chain 10`, one launch of 10
# trajectories, cold L2: 25.38 MB read + 4.36 MB written).
TRAFFIC = {"kernel": "k_chain_mixed", "kernel_rev": 15, "bytes_per_trajectory": 2974362}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# launches of the pipe probes sized to ~5 ms each on this GPU
PROBE_ITERS = {"ffma": 5000, "ffma2": 5000, "ex2": 600, "lds": 2500, "dfma": 75}


def measure_pipe_peaks(ctx, rsv, torch):
    """On-chip peaks the trajectory kernels are bound by, measured here: each
    rsv_pipe_probe launch keeps one unit busy on every SM; its operations /
    its CUDA-event time, best of 3 after one warm-up.  Units: op/s (an FMA is
    one operation), bytes/s for shared-memory loads."""
    out = {}
    for kind, it in PROBE_ITERS.items():
        best = None
        for r in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ops = rsv.rsv_pipe_probe(ctx, kind, it)
            b.record()
            b.synchronize()
            if r:
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
        out[kind] = ops / (best * 1e-3)
    out["fp32"] = max(out["ffma"], out["ffma2"])
    out["how"] = ("rsv_pipe_probe: 152 x 4 blocks of 512 threads, 8 independent chains per "
                  "thread of one instruction kind; operations / CUDA-event time, best of 3")
    return out


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def _barrier_max(ws, value):
    """The maximum of `value` over the ranks (the job's time is its slowest
    replica's)."""
    import torch
    if ws == 1:
        return value
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def replica_data_seed(rank: int) -> int:
    """Seed of the synthetic series of one replica: the replicas are independent
    chains on independent data (no data-path exchange between ranks)."""
    return SEED_DATA + 1000 * rank


def job_rate(ws: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return ws * units_per_rank / seconds_max


def cpu_baseline(budget_s: float = 12.0):
    """The FP64 oracle on this host, single thread, on trajectories of the same
    workload (T = 2^20, 100 x 0.005) until about budget_s of CPU work."""
    import oracle
    from paper_1603_08114_gb300 import synth
    s = synth.rsv_series(T_SITES, synth.THETA_STD, seed=SEED_DATA)
    h = s.h_true.copy()
    n = 0
    t0 = time.perf_counter()
    while True:
        r = oracle.chain(h, s.y, s.lnrv, s.theta, N_MD, DTAU, seed=7, n_traj=1, traj0=n)
        h = r["h"]
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 50:
            break
    # one trajectory of the small workload (T = 2000, 50 x 0.02) for scale
    s1 = synth.rsv_series(2000, synth.THETA_STD, seed=0)
    t1 = time.perf_counter()
    oracle.chain(s1.h_true, s1.y, s1.lnrv, s1.theta, 50, 0.02, seed=7, n_traj=20)
    small_s = (time.perf_counter() - t1) / 20
    return {"value": T_SITES * N_MD * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} FP64 oracle trajectories of the same workload (T=2^20, 100 x 0.005), "
                      f"{el:.1f} s, single-threaded C",
            "s_per_trajectory": {"T=2^20, 100 x 0.005": el / n, "T=2000, 50 x 0.02": small_s},
            "host": _host()}


def _host():
    """CPU model and logical core count of this host."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model name"):
                    model = v.strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            import subprocess
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"cpu": model or platform.machine(), "nproc": os.cpu_count()}


# The headline's trajectory shape: the step size and step count the tuner
# picks for the learned mass in every run so far (the largest step of its
# ladder that reaches 0.8 acceptance); the reference arm times the oracle on
# it, with a fixed diagonal mass of the learned mass's shape in its place.
HEAD_NMD, HEAD_DTAU = 78, 0.035


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores on the
    headline's trajectory shape (T = 2^20, 78 x 0.035, theta sampled, a fixed
    diagonal mass m ~ 30 in place of the learned one), each step one
    trajectory (a bounded sample of one 200-trajectory step)."""
    import oracle
    from paper_1603_08114_gb300 import synth
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s = synth.rsv_series(T_SITES, synth.THETA_STD, seed=SEED_DATA)
    minv = 1.0 / (30.0 + 3.0 * np.random.default_rng(3).random(T_SITES))
    h = s.h_true.copy()
    th = s.theta
    k = 0

    def one(h, th, k):
        r = oracle.chain(h, s.y, s.lnrv, th, HEAD_NMD, HEAD_DTAU, seed=7, n_traj=1, traj0=k,
                         update_theta=True, minv=minv)
        return r["h"], r["theta"]

    for _ in range(args.warmup):
        h, th = one(h, th, k)
        k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h, th = one(h, th, k)
        k += 1
    el = time.perf_counter() - t0
    v = T_SITES * HEAD_NMD * args.steps / el
    sample = (f"1 FP64 oracle trajectory (T=2^20, {HEAD_NMD} x {HEAD_DTAU}, theta sampled, fixed "
              f"diagonal mass m ~ 30) per step, single-threaded C")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": T_SITES, "n_md": HEAD_NMD, "dtau": HEAD_DTAU,
                   "traj_per_step": N_TRAJ, "precision": "fp64",
                   "mass": "diagonal m ~ 30 (fixed, the learned mass's shape)",
                   "l2": "host", "parallelism": f"replicas{ws}",
                   "step": "1 trajectory (a bounded sample of the 200-trajectory step)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host": _host()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


def run_ours(args):
    import torch

    from paper_1603_08114_gb300 import rsv, synth

    ws, rank, local = _dist()
    dev = torch.device("cuda", local)
    ctx = rsv.Context(local)
    s = synth.rsv_series(T_SITES, synth.THETA_STD, seed=replica_data_seed(rank))
    y = torch.tensor(s.y, device=dev)
    lnrv = torch.tensor(s.lnrv, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    snaps = torch.empty(N_TRAJ, T_SITES, dtype=torch.float32, device=dev)
    acc = torch.empty(N_TRAJ, dtype=torch.int32, device=dev)
    dH = torch.empty(N_TRAJ, dtype=torch.float64, device=dev)
    rsv.rsv_reserve(ctx, T_SITES)
    pipe = measure_pipe_peaks(ctx, rsv, torch)
    minv = None
    if args.mass_file:
        minv = torch.tensor(np.load(args.mass_file).astype(np.float32), device=dev)

    def run_chain(prec, mass, n_md, dtau, sampler, h, th, traj, rec=None):
        """One step: N_TRAJ trajectories, each followed by a theta sweep; rec =
        (snapshots [N_TRAJ][T], theta records [N_TRAJ][5], accept [N_TRAJ])."""
        sn, tho, ac = rec if rec is not None else (None, None, None)
        if sampler is not None:
            sampler.run(h, y, lnrv, th, N_TRAJ, seed=11 + rank, traj0=traj, snaps=sn,
                        theta_out=tho, accept_out=ac)
        else:
            rsv.rsv_hmc_chain(ctx, h, y, lnrv, th, n_md, dtau, N_TRAJ, prec=prec, minv=mass,
                              seed=11 + rank, traj0=traj, snaps=sn, thin=1, accept_out=ac,
                              update_theta=True, theta_out=tho)

    def site_moments(snaps_all):
        """Per-site posterior mean and variance of h over the chain with their
        Monte-Carlo standard errors by batch means (sqrt(n) batches of
        consecutive draws; the variance's from the batch means of the squared
        deviations): they include the slow theta direction that a per-site
        ESS from the leading autocorrelations would miss."""
        n = snaps_all.shape[0]
        nb = max(2, int(n ** 0.5))
        bl = n // nb
        bm = torch.empty(nb, T_SITES, dtype=torch.float64, device=dev)
        for b in range(nb):
            bm[b] = snaps_all[b * bl:(b + 1) * bl].double().mean(0)
        m = bm.mean(0)
        bq = torch.empty_like(bm)
        for b in range(nb):
            bq[b] = ((snaps_all[b * bl:(b + 1) * bl].double() - m) ** 2).mean(0)
        v = bq.mean(0)
        return dict(mean=m, var=v, mcse_mean=bm.std(0) / nb ** 0.5,
                    mcse_var=bq.std(0) / nb ** 0.5, batches=nb)

    def arm(prec, mass, warmup, steps, clocks=None, timing=False, n_md=N_MD, dtau=DTAU,
            sampler=None, moments=False, nvtx=False):
        # the chain starts from the generator's latent path, a posterior-typical
        # state (from lnRV - xi the first trajectories are all rejected); every
        # trajectory is followed by a Gibbs sweep of theta.  The warm-up steps
        # are its burn-in; ESS is taken over the whole timed chain (steps x
        # N_TRAJ draws), after the timed region.
        h = torch.tensor(s.h_true, device=dev)
        th = torch.tensor(s.theta, dtype=torch.float64, device=dev)
        traj = 0
        for _ in range(warmup):
            run_chain(prec, mass, n_md, dtau, sampler, h, th, traj)
            traj += N_TRAJ
        nonfinite = rsv.rsv_sync_status(ctx, allow_nonfinite=True) == rsv.RSV_ENONFINITE
        n_all = steps * N_TRAJ
        snaps_all = torch.empty(n_all, T_SITES, dtype=torch.float32, device=dev)
        thetas_all = torch.empty(n_all, 5, dtype=torch.float64, device=dev)
        acc_all = torch.empty(n_all, dtype=torch.int32, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        rsv.rsv_stats(ctx, reset=True)
        rsv.rsv_timing(ctx, timing)
        _barrier(ws)
        if clocks:
            clocks.__enter__()
        if nvtx:  # marks the headline's timed kernels for ncu (--nvtx-include "timed/")
            torch.cuda.nvtx.range_push("timed")
        launches = 0
        md0 = sampler.md_steps if sampler is not None else 0
        for k in range(steps):
            flush.zero_()
            l0 = rsv.rsv_stats(ctx, reset=False)[0]
            sl = slice(k * N_TRAJ, (k + 1) * N_TRAJ)
            ev[k][0].record()
            run_chain(prec, mass, n_md, dtau, sampler, h, th, traj,
                      (snaps_all[sl], thetas_all[sl], acc_all[sl]))
            ev[k][1].record()
            traj += N_TRAJ
            launches += rsv.rsv_stats(ctx, reset=False)[0] - l0
        if nvtx:
            torch.cuda.nvtx.range_pop()
        _barrier(ws)
        if clocks:
            clocks.__exit__()
        rsv.rsv_timing(ctx, False)
        _, traj_launches, traj_ms = rsv.rsv_stats(ctx, reset=True)
        # a non-finite dH is a rejected trajectory, not a failure; it is reported
        nonfinite |= rsv.rsv_sync_status(ctx, allow_nonfinite=True) == rsv.RSV_ENONFINITE
        ms = [a.elapsed_time(b) for a, b in ev]
        total_s = _barrier_max(ws, sum(ms) / 1e3)
        sec_per_step = total_s / steps
        # leapfrog steps per site actually run per step (the mass sampler may
        # have fallen back to the plain settings part-way)
        md_per_step = ((sampler.md_steps - md0) / steps if sampler is not None
                       else n_md * N_TRAJ)
        ess = rsv.rsv_ess(ctx, snaps_all)
        ess_th = rsv.rsv_ess(ctx, thetas_all.float().contiguous()).cpu().numpy()
        ess_med, ess_min = float(ess.median()), float(ess.min())
        mom = site_moments(snaps_all) if moments else None
        del snaps_all
        return dict(
            site_updates_per_s=job_rate(ws, T_SITES * md_per_step, sec_per_step),
            md_steps_per_step=md_per_step,
            n_md=n_md, dtau=dtau,
            ms_per_step=1e3 * sec_per_step, timed_s=total_s, draws=n_all,
            ess_h_median_per_s=ws * ess_med / total_s,
            ess_h_min_per_s=ws * ess_min / total_s,
            ess_h_median=ess_med, ess_h_min=ess_min,
            ess_theta_per_s={n: ws * float(v) / total_s for n, v in zip(THETA_NAMES, ess_th)},
            ess_theta={n: float(v) for n, v in zip(THETA_NAMES, ess_th)},
            accept_rate=float(acc_all.float().mean()),
            launches=launches, traj_launches=traj_launches, traj_ms=traj_ms,
            nonfinite_dH_seen=bool(nonfinite), moments=mom, h_end=h, theta_end=th)

    def step_kernel_us(yv, lv, h0, n_hi, n=10):
        """Per-step time of the mixed trajectory kernel (identity mass, theta
        fixed): its time at n_hi steps minus at one step, on the tiling the
        library picks for n_hi, per extra step; and its time at one step."""
        pl = rsv.Plan(ctx, np.array([0, T_SITES], dtype=np.int64), n_hi, "mixed")
        pi = pl.info()
        pl.close()
        nt_, j_ = pi["threads"], pi["sites_per_thread"]
        rsv.rsv_set_schedule(ctx, nt_, j_, nt_ * j_ - 2 * (n_hi + 1) - 3)
        rsv.rsv_set_persistent(ctx, False)  # the per-trajectory kernels, compared alike
        out = []
        try:
            for n_md in (n_hi, 1):
                hh = torch.tensor(h0, device=dev)
                th = torch.tensor(s.theta, dtype=torch.float64, device=dev)
                rsv.rsv_hmc_chain(ctx, hh, yv, lv, th, n_md, DTAU, 2, prec="mixed", seed=77)
                torch.cuda.synchronize()
                rsv.rsv_stats(ctx, reset=True)
                rsv.rsv_timing(ctx, True)
                rsv.rsv_hmc_chain(ctx, hh, yv, lv, th, n_md, DTAU, n, prec="mixed", seed=78,
                                  traj0=2)
                torch.cuda.synchronize()
                rsv.rsv_timing(ctx, False)
                _, nl, ms = rsv.rsv_stats(ctx, reset=True)
                out.append(1e3 * ms / max(nl, 1))
        finally:
            rsv.rsv_set_schedule(ctx)
            rsv.rsv_set_persistent(ctx, True)
        return (out[0] - out[1]) / (n_hi - 1), out[1], {"threads": nt_, "sites_per_thread": j_}

    def leverage_leg(steps):
        """The RSV model with leverage, rho = corr(eps_t, eta_t) = RHO_STD, on a
        2^20-site series drawn from it: mixed, identity mass, 100 x 0.005, theta
        fixed at its true value (the theta update is for rho = 0).  Chain rate,
        ESS of h, and the step time of the leverage kernel against the plain
        one (same series, rho = 0) on one tiling."""
        sl = synth.rsv_series_leverage(T_SITES, synth.THETA_STD, synth.RHO_STD,
                                       seed=SEED_DATA + 7 + 1000 * rank)
        yl, ll = torch.tensor(sl.y, device=dev), torch.tensor(sl.lnrv, device=dev)
        rsv.rsv_set_leverage(ctx, synth.RHO_STD)
        try:
            h = torch.tensor(sl.h_true, device=dev)
            th = torch.tensor(sl.theta, dtype=torch.float64, device=dev)
            traj = 0
            for _ in range(2):
                rsv.rsv_hmc_chain(ctx, h, yl, ll, th, N_MD, DTAU, N_TRAJ, prec="mixed",
                                  seed=21 + rank, traj0=traj)
                traj += N_TRAJ
            rsv.rsv_sync_status(ctx)
            ms, ess_med, ess_min, rates = [], [], [], []
            for _ in range(steps):
                flush.zero_()
                a_ev = torch.cuda.Event(enable_timing=True)
                b_ev = torch.cuda.Event(enable_timing=True)
                a_ev.record()
                rsv.rsv_hmc_chain(ctx, h, yl, ll, th, N_MD, DTAU, N_TRAJ, prec="mixed",
                                  seed=21 + rank, traj0=traj, snaps=snaps, thin=1,
                                  accept_out=acc)
                b_ev.record()
                traj += N_TRAJ
                e = rsv.rsv_ess(ctx, snaps)
                ess_med.append(float(e.median()))
                ess_min.append(float(e.min()))
                rates.append(float(acc.float().mean()))
                ms.append(a_ev.elapsed_time(b_ev))
            rsv.rsv_sync_status(ctx)
            sec = _barrier_max(ws, sum(ms) / 1e3) / steps
            us_lev, us_lev1, sched = step_kernel_us(yl, ll, sl.h_true, N_MD)
        finally:
            rsv.rsv_set_leverage(ctx, 0.0)
        us_plain, us_plain1, _ = step_kernel_us(yl, ll, sl.h_true, N_MD)
        return {"rho": synth.RHO_STD, "T": T_SITES, "n_md": N_MD, "dtau": DTAU,
                "theta": "fixed (true value)", "precision": "mixed", "mass": "identity",
                "site_updates_per_s": ws * T_SITES * N_MD * N_TRAJ / sec,
                "ms_per_step": 1e3 * sec, "traj_per_step": N_TRAJ,
                "ess_h_median_per_s": ws * statistics.mean(ess_med) / sec,
                "ess_h_min_per_s": ws * statistics.mean(ess_min) / sec,
                "accept_rate": statistics.mean(rates),
                "kernel_us_per_step": us_lev, "kernel_us_one_step": us_lev1,
                "plain_kernel_us_per_step": us_plain, "plain_kernel_us_one_step": us_plain1,
                "schedule": sched,
                "how": "chain: CUDA events around each step of N trajectories (L2 flushed); "
                       "kernel: k_traj_mixed time at n_md minus at n_md = 1, per step"}

    def batched_leg(steps):
        """The 4096-series workload: one persistent launch per trajectory of all
        series, autotuned block shape, replayed from a CUDA graph."""
        from paper_1603_08114_gb300 import autotune
        b = synth.rsv_batch(4096, 500, 8192, seed=2)
        n = len(b.offsets) - 1
        N = int(b.offsets[-1])
        yb, lb = torch.tensor(b.y, device=dev), torch.tensor(b.lnrv, device=dev)
        thb = torch.tensor(b.theta.ravel(), device=dev)
        h0 = torch.tensor(b.h_true, device=dev)
        hb = h0.clone()
        rsv.rsv_reserve(ctx, max(N, T_SITES), n)
        plan, sched = autotune.tune_plan(ctx, b.offsets, 50, "mixed", yb, lb, thb, 0.02, h0)
        per_graph = 10  # trajectories of every series per graph replay
        accb = torch.empty(per_graph * n, dtype=torch.int32, device=dev)
        rsv.rsv_hmc_batched(ctx, plan, hb, yb, lb, thb, 0.02, seed=3, traj0=0, n_traj=per_graph,
                            accept_out=accb)
        torch.cuda.synchronize()
        stream = torch.cuda.Stream()
        graphs = []
        with torch.cuda.stream(stream):
            for k in range(steps + 3):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    rsv.rsv_hmc_batched(ctx, plan, hb, yb, lb, thb, 0.02, seed=3,
                                        traj0=per_graph * (1 + k), n_traj=per_graph,
                                        accept_out=accb)
                graphs.append(g)
        for g in graphs[:3]:
            g.replay()
        torch.cuda.synchronize()
        rates = []
        ms = 0.0
        for g in graphs[3:]:
            flush.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            c.record()
            c.synchronize()
            ms += a.elapsed_time(c)
            rates.append(float(accb.float().mean()))
        rsv.rsv_sync_status(ctx)
        info = plan.info()
        plan.close()
        ntr = per_graph * steps
        return {"site_updates_per_s": N * 50 * ntr / (ms / 1e3), "ms_per_trajectory": ms / ntr,
                "series": n, "sites": N, "n_md": 50, "dtau": 0.02, "precision": "mixed",
                "accept_rate": statistics.mean(rates), "graph": True,
                "trajectories_per_graph": per_graph,
                "schedule": {"threads": sched["threads"], "sites_per_thread":
                             sched["sites_per_thread"], "cached": sched["cached"], **info}}

    def c1_leg():
        """The T = 2000 workload: plain FP64 HMC, theta held at its true values,
        1000 trajectories of 50 x 0.02 in one rsv_hmc_chain call (seed 0
        series, Philox momenta and uniforms); two calls, the second timed."""
        sc = synth.rsv_series(2000, synth.THETA_STD, seed=0)
        yc, lc = torch.tensor(sc.y, device=dev), torch.tensor(sc.lnrv, device=dev)
        hc = torch.tensor(sc.h_true, device=dev)
        thc = torch.tensor(sc.theta, dtype=torch.float64, device=dev)
        n = 1000
        snc = torch.empty(n, 2000, dtype=torch.float32, device=dev)
        acc_c = torch.empty(n, dtype=torch.int32, device=dev)
        rsv.rsv_hmc_chain(ctx, hc, yc, lc, thc, 50, 0.02, n, prec="fp64", seed=41)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rsv.rsv_hmc_chain(ctx, hc, yc, lc, thc, 50, 0.02, n, prec="fp64", seed=41, traj0=n,
                          snaps=snc, thin=1, accept_out=acc_c)
        b.record()
        b.synchronize()
        rsv.rsv_sync_status(ctx)
        sec = _barrier_max(ws, a.elapsed_time(b) / 1e3)
        e = rsv.rsv_ess(ctx, snc)
        return {"T": 2000, "n_md": 50, "dtau": 0.02, "trajectories": n, "precision": "fp64",
                "theta": "held at its true values", "site_updates_per_s": ws * 2000 * 50 * n / sec,
                "ms_per_1000_trajectories": 1e3 * sec,
                "ess_h_median_per_s": ws * float(e.median()) / sec,
                "ess_h_min_per_s": ws * float(e.min()) / sec,
                "accept_rate": float(acc_c.float().mean())}

    def c4_leg(n_cmp=10, n_rate=20):
        """T = 2^22 (phi 0.97, s_eta^2 0.03, seed 3), 100 x 0.003: the mixed
        path's rate (a chain of n_rate trajectories, theta fixed) and its
        error against the FP64 GPU path (itself at 1e-12 of the FP64 oracle in
        the tests) on n_cmp trajectories from the same start, momenta and
        uniforms: h' error, dH error, accept agreement."""
        T4 = 1 << 22
        s4 = synth.rsv_series(T4, synth.THETA_LARGE, seed=3)
        y4, l4 = torch.tensor(s4.y, device=dev), torch.tensor(s4.lnrv, device=dev)
        rsv.rsv_reserve(ctx, T4)
        h4 = torch.tensor(s4.h_true, device=dev)
        th4 = torch.tensor(s4.theta, dtype=torch.float64, device=dev)
        rsv.rsv_hmc_chain(ctx, h4, y4, l4, th4, 100, 0.003, 2, prec="mixed", seed=51)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        acc4 = torch.empty(n_rate, dtype=torch.int32, device=dev)
        a.record()
        rsv.rsv_hmc_chain(ctx, h4, y4, l4, th4, 100, 0.003, n_rate, prec="mixed", seed=51,
                          traj0=2, accept_out=acc4)
        b.record()
        b.synchronize()
        sec = _barrier_max(ws, a.elapsed_time(b) / 1e3)
        err_h, err_dh, agree, marginal = 0.0, 0.0, 0, 0
        for k in range(n_cmp):
            p0 = torch.tensor(synth.standard_normals(T4, 300 + k), device=dev)
            lu = torch.tensor(synth.log_uniforms(1, 400 + k), device=dev)
            out = {}
            for prec in ("fp64", "mixed"):
                hh, pp = h4.clone(), p0.clone()
                dHk, ak = rsv.rsv_hmc_trajectory(ctx, hh, pp, y4, l4, s4.theta, 100, 0.003,
                                                 prec=prec, log_u=lu)
                out[prec] = (hh, float(dHk.item()), int(ak.item()))
            (h64, d64, a64), (h32, d32, a32) = out["fp64"], out["mixed"]
            if a64 and a32:
                err_h = max(err_h, float(((h32 - h64).abs() / h64.abs().clamp(min=1.0)).max()))
            err_dh = max(err_dh, abs(d32 - d64))
            if abs(d64 + float(lu.item())) > 1e-2:
                agree += int(a64 == a32)
            else:
                marginal += 1
        rsv.rsv_sync_status(ctx)
        return {"T": T4, "n_md": 100, "dtau": 0.003, "theta": list(synth.THETA_LARGE),
                "precision": "mixed (FP32 leapfrog, double-float dH)",
                "site_updates_per_s": ws * T4 * 100 * n_rate / sec,
                "ms_per_trajectory": 1e3 * sec / n_rate,
                "accept_rate": float(acc4.float().mean()),
                "vs_fp64_gpu": {"trajectories": n_cmp, "h_rel_err_max": err_h,
                                "dH_abs_err_max": err_dh, "accept_agree": agree,
                                "accept_compared": n_cmp - marginal,
                                "marginal_skipped": marginal,
                                "bounds": {"h": 1e-4, "dH": 1e-3, "gap": 1e-2}}}

    def c5_compare(head_r, ident_r):
        """Learned vs identity mass at equal posterior accuracy: per-site
        posterior means and variances of the two timed chains agree within
        their combined Monte-Carlo errors (z = |difference| / combined MCSE;
        under equal moments about 0.05 % of 2^20 sites exceed 3.5)."""
        a, b = head_r["moments"], ident_r["moments"]
        if a is None or b is None:
            return None
        z_m = (a["mean"] - b["mean"]).abs() / torch.sqrt(a["mcse_mean"] ** 2 + b["mcse_mean"] ** 2)
        z_v = (a["var"] - b["var"]).abs() / torch.sqrt(a["mcse_var"] ** 2 + b["mcse_var"] ** 2)
        q = torch.tensor([0.5, 0.999], dtype=torch.float64, device=dev)
        # under equal moments z is about Student-t with (batches - 1) degrees of
        # freedom (each MCSE from sqrt(n) batch means)
        dof = min(a["batches"], b["batches"]) - 1
        try:
            from scipy import stats as sps
            expected = float(2 * sps.t.sf(3.5, dof))
        except ImportError:
            expected = 4.65e-4
        return {"sites": T_SITES,
                "mean_z_median_p999": [float(v) for v in torch.quantile(z_m[::8], q)],
                "mean_frac_z_over_3.5": float((z_m > 3.5).double().mean()),
                "var_z_median_p999": [float(v) for v in torch.quantile(z_v[::8], q)],
                "var_frac_z_over_3.5": float((z_v > 3.5).double().mean()),
                "expected_frac_z_over_3.5": expected,
                "batches": [a["batches"], b["batches"]],
                "how": "per-site mean and variance of h over each arm's whole timed chain; "
                       "MCSE by batch means with sqrt(n) batches (the variance's from the "
                       "squared deviations); z = |difference| / combined MCSE"}

    # headline: mixed precision (diagonal mass when given)
    # learned diagonal mass (untimed set-up): moments of the plain sampler over
    # n_snap trajectories, 2000 Adam steps, inverse mass, step tuned to ~0.8
    # acceptance at the plain sampler's physical trajectory length (0.5 sqrt(m)
    # in the mass's time units, m the median mass: with p ~ N(0, m) a site
    # moves at ~1/sqrt(m) per unit time); fallback to the plain sampler below
    # 0.6 acceptance
    learned_info, sampler, head_nmd, head_dt = None, None, N_MD, DTAU
    mass_length = None
    if minv is None and not args.no_learned:
        from paper_1603_08114_gb300 import learned
        h0 = torch.tensor(s.h_true, device=dev)
        th0 = torch.tensor(s.theta, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        mean, m2, cnt = learned.collect_moments(ctx, h0, y, lnrv, th0, args.n_snap, N_MD, DTAU,
                                                seed=5 + rank)
        torch.cuda.synchronize()
        t_snap = time.perf_counter() - t0
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record()
        tm = learned.train_mass(ctx, y, lnrv, s.theta, mean, m2, cnt, steps=2000, batch=4096,
                                lr=1e-3, seed=7 + rank)
        b_ev.record()
        b_ev.synchronize()
        m_med = float(torch.quantile((1.0 / tm.minv[::16]).float(), 0.5))
        mass_length = N_MD * DTAU * m_med ** 0.5
        t1 = time.perf_counter()
        head_dt, head_nmd = learned.tune_step(ctx, h0, y, lnrv, th0, tm.minv, length=mass_length)
        torch.cuda.synchronize()
        t_tune = time.perf_counter() - t1
        minv = tm.minv
        # one window per step: the mass's acceptance is checked once per 200
        # trajectories, and a step is one chain call
        sampler = learned.MassSampler(ctx, minv, head_dt, head_nmd, DTAU, N_MD, window=N_TRAJ)
        m = (1.0 / minv).float()
        losses = tm.losses.cpu().numpy()
        learned_info = {"snapshots": int(cnt), "snapshot_s": t_snap,
                        "train_steps": 2000, "train_ms": a_ev.elapsed_time(b_ev),
                        "loss_first": float(losses[:10].mean()),
                        "loss_last": float(losses[-50:].mean()),
                        "m_quantiles": [float(v) for v in torch.quantile(
                            m[::16], torch.tensor([0.01, 0.5, 0.99], device=dev))],
                        "tune_s": t_tune,
                        "setup_s": t_snap + a_ev.elapsed_time(b_ev) / 1e3 + t_tune,
                        "dtau": head_dt, "n_md": head_nmd, "trajectory_length": mass_length}

    if minv is not None and mass_length is None:  # a mass from --mass-file
        mass_length = N_MD * DTAU * float(torch.quantile((1.0 / minv[::16]).float(), 0.5)) ** 0.5
    clocks = Clocks(local)
    head = arm("mixed", minv, args.warmup, args.steps, clocks=clocks, timing=True,
               n_md=head_nmd, dtau=head_dt, sampler=sampler, moments=minv is not None,
               nvtx=True)
    if learned_info is not None:
        learned_info["fell_back"] = bool(sampler.fell_back)
        learned_info["window_accept"] = [round(r, 3) for r in sampler.history]
    # comparisons: plain mixed and plain FP64 samplers (identity mass, 100 x 0.005)
    ident = fp64 = batched = mn = mn4 = levr = c1 = c4 = t2gpu = c5 = None
    if args.only != "mixed":
        if minv is not None:
            # the same chain length as the headline: the moment comparison
            # needs both chains to have explored theta alike
            ident = arm("mixed", None, min(args.warmup, 3), args.steps, moments=True)
            c5 = c5_compare(head, ident)
        fp64 = arm("fp64", None, min(args.warmup, 3), min(args.steps, 3), timing=True)
        batched = batched_leg(max(3, min(args.steps, 10)))
        levr = leverage_leg(min(args.steps, 3))
        c1 = c1_leg()
        c4 = c4_leg()
        t2gpu = table2_gpu(ctx, rsv, synth, torch, TABLE2_B_SHORT)
        # the minimum-norm integrator (two forces per step) at the plain
        # sampler's physical trajectory length (0.5; 0.5 sqrt(m) in the
        # learned mass's units):
        # the fewest steps whose acceptance over 40 trial trajectories
        # reaches 0.8, identity mass and learned mass
        def tune_mn(mass, length, tries):
            h_t = torch.tensor(s.h_true, device=dev)
            th_t = torch.tensor(s.theta, dtype=torch.float64, device=dev)
            acc_t = torch.empty(40, dtype=torch.int32, device=dev)
            for n_try in tries:
                rsv.rsv_hmc_chain(ctx, h_t.clone(), y, lnrv, th_t.clone(), n_try, length / n_try,
                                  40, prec="mixed", minv=mass, seed=123, accept_out=acc_t)
                if float(acc_t.float().mean()) >= 0.8:
                    return n_try
            return tries[-1]
        mn, mn4 = {}, {}
        for integ, out, tries in (("omelyan2", mn, (3, 4, 5, 6, 8, 10, 12, 15, 20, 30)),
                                  ("omelyan4", mn4, (2, 3, 4, 5, 6, 8, 10, 15))):
            rsv.rsv_set_integrator(ctx, integ)
            try:
                for tag, mass, length in (("identity", None, N_MD * DTAU),
                                          ("learned", minv, mass_length)):
                    if tag == "learned" and mass is None:
                        continue
                    n_mn = tune_mn(mass, length, tries)
                    r = arm("mixed", mass, min(args.warmup, 3), min(args.steps, 3), n_md=n_mn,
                            dtau=length / n_mn)
                    r["n_md"], r["dtau"] = n_mn, length / n_mn
                    out[tag] = r
            finally:
                rsv.rsv_set_integrator(ctx, "leapfrog")

    # end to end through the public API with host buffers: the headline's own
    # call (the same sampler, snapshots and theta records), its inputs (the
    # chain state h and theta carried on the host between steps, y, lnRV)
    # copied from pinned memory before and its results (h', theta and accept
    # records) copied back after, every step inside the timed region; L2
    # flushed between steps outside it, as for `value`
    import dataclasses
    e2e_sampler = dataclasses.replace(sampler, history=[], md_steps=0) if sampler else None
    h_host = torch.tensor(s.h_true).pin_memory()
    y_host = torch.tensor(s.y).pin_memory()
    l_host = torch.tensor(s.lnrv).pin_memory()
    th_host = torch.tensor(s.theta, dtype=torch.float64).pin_memory()
    out_th = torch.empty(N_TRAJ, 5, dtype=torch.float64).pin_memory()
    out_a = torch.empty(N_TRAJ, dtype=torch.int32).pin_memory()
    hd = torch.empty(T_SITES, dtype=torch.float64, device=dev)
    yd = torch.empty_like(hd)
    ld = torch.empty_like(hd)
    thd = torch.empty(5, dtype=torch.float64, device=dev)
    th_rec = torch.empty(N_TRAJ, 5, dtype=torch.float64, device=dev)
    e2e_steps = max(1, min(args.steps, 5))
    e2e_ms, e2e_md = 0.0, 0
    _barrier(ws)
    for k in range(e2e_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        md0 = e2e_sampler.md_steps if e2e_sampler else 0
        e0.record()
        hd.copy_(h_host, non_blocking=True)
        yd.copy_(y_host, non_blocking=True)
        ld.copy_(l_host, non_blocking=True)
        thd.copy_(th_host, non_blocking=True)
        if e2e_sampler is not None:
            e2e_sampler.run(hd, yd, ld, thd, N_TRAJ, seed=99 + rank, traj0=k * N_TRAJ,
                            snaps=snaps, theta_out=th_rec, accept_out=acc)
        else:
            rsv.rsv_hmc_chain(ctx, hd, yd, ld, thd, head_nmd, head_dt, N_TRAJ, prec="mixed",
                              minv=minv, seed=99 + rank, traj0=k * N_TRAJ, snaps=snaps, thin=1,
                              accept_out=acc, update_theta=True, theta_out=th_rec)
        h_host.copy_(hd, non_blocking=True)
        th_host.copy_(thd, non_blocking=True)
        out_th.copy_(th_rec, non_blocking=True)
        out_a.copy_(acc, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_md += (e2e_sampler.md_steps - md0) if e2e_sampler else head_nmd * N_TRAJ
    e2e_s = _barrier_max(ws, e2e_ms / 1e3)
    h2d = 3 * T_SITES * 8 + 5 * 8
    d2h = T_SITES * 8 + 5 * 8 + N_TRAJ * (5 * 8 + 4)

    # MD-only rate (the paper's elementary step): trajectory-kernel time at the
    # headline length minus that at one step, per leapfrog step, no theta update
    def kernel_us(n_md, n=10):
        hh = torch.tensor(s.h_true, device=dev)
        th = torch.tensor(s.theta, dtype=torch.float64, device=dev)
        rsv.rsv_hmc_chain(ctx, hh, y, lnrv, th, n_md, head_dt, 2, prec="mixed", minv=minv,
                          seed=77)
        torch.cuda.synchronize()
        rsv.rsv_stats(ctx, reset=True)
        rsv.rsv_timing(ctx, True)
        rsv.rsv_hmc_chain(ctx, hh, y, lnrv, th, n_md, head_dt, n, prec="mixed", minv=minv,
                          seed=78, traj0=2)
        torch.cuda.synchronize()
        rsv.rsv_timing(ctx, False)
        _, nl, ms = rsv.rsv_stats(ctx, reset=True)
        return 1e3 * ms / max(nl, 1)
    # both lengths on the headline's tiling (its halo for n_md): the shape a
    # chain call of the headline uses, its tile fixed for the one-step run too
    cs = rsv.rsv_chain_schedule(ctx, T_SITES, head_nmd, "mixed", with_mass=minv is not None)
    nt_, j_ = cs["threads"], cs["sites_per_thread"]
    rsv.rsv_set_schedule(ctx, nt_, j_, nt_ * j_ - 2 * (head_nmd + 1) - 3)
    t_hi, t_lo = kernel_us(head_nmd), kernel_us(1)
    rsv.rsv_set_schedule(ctx)
    per_step_us = (t_hi - t_lo) / max(head_nmd - 1, 1)
    md = {"site_updates_per_s": ws * T_SITES / (per_step_us * 1e-6), "unit": UNIT,
          "us_per_step": per_step_us, "us_per_trajectory_fixed": t_lo - per_step_us,
          "kernel_us_per_trajectory": t_hi, "n_md": head_nmd,
          "schedule": {"threads": nt_, "sites_per_thread": j_,
                       "persistent": cs["persistent"]},
          "how": "trajectory time of the chain kernel at n_md minus at n_md = 1, per step "
                 "(CUDA events around a 10-trajectory chain call)"}

    # roofline of the headline's trajectory kernel: the method's algorithmic
    # work (ALG_OPS FP32 operations + 1 exp per site and leapfrog step) over
    # the launch's event time, against the FP32 and ex2 peaks measured above
    per_launch_s = head["traj_ms"] / 1e3 / max(head["traj_launches"], 1)
    site_steps = T_SITES * head_nmd
    achieved = ALG_OPS_PER_SITE_STEP * site_steps / per_launch_s
    fp32_peak = pipe["fp32"]
    ex2_rate = site_steps / per_launch_s
    # DRAM bytes (read + write) of one headline launch from the ncu capture in
    # profiles/, valid only for the kernel revision it was taken on
    from paper_1603_08114_gb300 import autotune as _at
    traffic = (TRAFFIC["bytes_per_trajectory"] if TRAFFIC["kernel_rev"] == _at.KERNEL_REV
               else None)
    fp64_roof = None
    if fp64 is not None:
        f_launch = fp64["traj_ms"] / 1e3 / max(fp64["traj_launches"], 1)
        fp64_ach = ALG_OPS_PER_SITE_STEP * T_SITES * N_MD / f_launch
        fp64_roof = {"bound": "fp64", "achieved": fp64_ach / 1e12, "peak": pipe["dfma"] / 1e12,
                     "unit": "Top/s", "frac": fp64_ach / pipe["dfma"],
                     "per_launch_ms": f_launch * 1e3, "peak_kind": "measured DFMA rate"}

    if rank == 0:
        cpu = cpu_baseline() if (ws == 1 and not args.no_cpu) else None
        t2 = None
        if t2gpu is not None:
            t2cpu = table2_cpu(TABLE2_B_SHORT) if (ws == 1 and not args.no_cpu) else None
            t2 = table2_summary(TABLE2_B_SHORT, t2gpu, t2cpu)

        def arm_summary(r, extra=None):
            if r is None:
                return None
            d = {"site_updates_per_s": r["site_updates_per_s"], "n_md": r["n_md"],
                 "dtau": r["dtau"], "ms_per_step": r["ms_per_step"], "draws": r["draws"],
                 "ess_h_median_per_s": r["ess_h_median_per_s"],
                 "ess_h_min_per_s": r["ess_h_min_per_s"],
                 "ess_theta_per_s": r["ess_theta_per_s"], "accept_rate": r["accept_rate"]}
            d.update(extra or {})
            return d

        learned_cmp = None
        if learned_info is not None and ident is not None:
            setup = learned_info["setup_s"]
            ess_l = head["ess_h_median_per_s"] * head["timed_s"]
            learned_cmp = {
                "ess_h_median_per_s": {"learned": head["ess_h_median_per_s"],
                                       "identity": ident["ess_h_median_per_s"]},
                "ess_theta_per_s": {"learned": head["ess_theta_per_s"],
                                    "identity": ident["ess_theta_per_s"]},
                "equal_posterior_moments": c5,
                "setup_s": setup,
                "learned_ess_h_median_per_s_with_setup_over_timed_chain":
                    ess_l / (head["timed_s"] + setup),
                "learned_ess_h_median_per_s_with_setup_over_1e5_trajectories":
                    ess_l / (head["timed_s"] + setup * head["draws"] / 1e5),
                "gain_h_median": head["ess_h_median_per_s"] / ident["ess_h_median_per_s"],
                "note": "the learned mass gains only if gain_h_median > 1: the posterior "
                        "variance of this workload is nearly the same at every site"}
        line = {
            "metric": METRIC, "value": head["site_updates_per_s"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "T": T_SITES, "n_md": head_nmd, "dtau": head_dt,
                       "traj_per_step": N_TRAJ, "precision": "mixed",
                       "mass": "learned" if minv is not None else "identity",
                       "l2": "flushed before every step (256 MB write, untimed)",
                       "parallelism": f"replicas{ws}"},
            "ess": {"h_median_per_s": head["ess_h_median_per_s"],
                    "h_min_per_s": head["ess_h_min_per_s"],
                    "h_median": head["ess_h_median"], "h_min": head["ess_h_min"],
                    "theta_per_s": head["ess_theta_per_s"], "theta": head["ess_theta"],
                    "draws": head["draws"], "accept_rate": head["accept_rate"],
                    "how": "Geyer ESS over the whole timed chain (steps x 200 draws) / the "
                           "chain's summed step time"},
            "fp64_plain": arm_summary(fp64, {"roofline": fp64_roof}),
            "mixed_identity": arm_summary(ident),
            "learned": learned_info,
            "learned_vs_identity": learned_cmp,
            "c1": c1, "c4": c4, "table2": t2,
            "batched": None if batched is None else dict(batched, roofline={
                "bound": "alu", "unit": "Top/s", "peak": fp32_peak / 1e12,
                "achieved": batched["site_updates_per_s"] * ALG_OPS_PER_SITE_STEP / 1e12,
                "frac": batched["site_updates_per_s"] * ALG_OPS_PER_SITE_STEP / fp32_peak,
                "how": "the method's 10 FP32 operations per site-step of all series over a "
                       "trajectory's time, against the measured FP32 FMA rate"}),
            "leverage": levr,
            "mixed_omelyan2": None if mn is None else {
                tag: arm_summary(r, {"integrator": "minimum-norm (Omelyan), 2 force "
                                                   "evaluations per step", "mass": tag,
                                     "force_evaluations_per_trajectory": 2 * r["n_md"]})
                for tag, r in mn.items()},
            "mixed_omelyan4": None if mn4 is None else {
                tag: arm_summary(r, {"integrator": "fourth-order minimum-norm (Omelyan), 4 "
                                                   "force evaluations per step", "mass": tag,
                                     "force_evaluations_per_trajectory": 4 * r["n_md"]})
                for tag, r in mn4.items()},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
                         "unit": "Top/s", "frac": achieved / fp32_peak, "traffic": traffic,
                         "kernel": "k_chain_mixed" if cs["persistent"] else "k_traj_mixed",
                         "per": "trajectory" if cs["persistent"] else "launch",
                         "peak_kind": "measured FP32 FMA rate (rsv_pipe_probe, the larger of "
                                      "FFMA and FFMA2), this run",
                         "per_launch_ms": per_launch_s * 1e3,
                         "algorithmic_ops_per_site_step": ALG_OPS_PER_SITE_STEP,
                         "site_steps_per_launch": site_steps,
                         "issued_ops_per_site_step": IMPL_OPS_PER_SITE_STEP_MIXED,
                         "issued_frac": achieved / fp32_peak * IMPL_OPS_PER_SITE_STEP_MIXED
                         / ALG_OPS_PER_SITE_STEP,
                         "ex2": {"achieved": ex2_rate / 1e12, "peak": pipe["ex2"] / 1e12,
                                 "frac": ex2_rate / pipe["ex2"]},
                         "md_only_frac": ALG_OPS_PER_SITE_STEP * T_SITES
                         / (md["us_per_step"] * 1e-6) / fp32_peak},
            "pipe_peaks": {"unit": "T op/s (lds: TB/s)",
                           **{k: (v / 1e12 if isinstance(v, float) else v)
                              for k, v in pipe.items()}},
            "cpu_baseline": cpu,
            "md_only": md,
            "e2e": {"value": ws * T_SITES * e2e_md / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": head["launches"],
            "clocks": clocks.summary(),
        }
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# The paper's Table 2 (Sec. 5): time of one elementary MD step (Kernels 1-3,
# one leapfrog step over all T sites), T = 512 B, fitted as f(B) = A + C B;
# GTX 760 (CUDA Fortran, FP32) and i7-4770.
PAPER_TABLE2 = {"gpu": {"A": 1.13e-5, "C": 2.25e-7}, "cpu": {"A": -1.42e-6, "C": 3.87e-6},
                "gain_limit": 17.2, "hardware": "GTX 760 / i7-4770 3.4 GHz, FP32"}
TABLE2_B = (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048)
TABLE2_B_SHORT = (1, 8, 64, 512, 2048)   # the ladder of the default run


def fit_linear(B, f):
    """Least-squares f(B) = A + C B; returns (A, C)."""
    B = np.asarray(B, dtype=np.float64)
    M = np.stack([np.ones_like(B), B], axis=1)
    (A, C), *_ = np.linalg.lstsq(M, np.asarray(f, dtype=np.float64), rcond=None)
    return float(A), float(C)


def table2_gpu(ctx, rsv, synth, torch, B_list, n_lo=10, n_hi=110):
    """Seconds per elementary MD step (one leapfrog step over all T = 512 B
    sites) of the mixed and FP64 trajectory kernels: the kernel's time at
    n_hi steps minus at n_lo on one tiling, over n_hi - n_lo (CUDA events)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    res = {"gpu_mixed": [], "gpu_fp64": []}
    for B in B_list:
        T = 512 * B
        s = synth.rsv_series(T, synth.THETA_STD, seed=1)
        y = torch.tensor(s.y, device=dev)
        lr = torch.tensor(s.lnrv, device=dev)
        for prec in ("mixed", "fp64"):
            cs = rsv.rsv_chain_schedule(ctx, T, n_hi, prec)
            nt, j = cs["threads"], cs["sites_per_thread"]
            if T > nt * j - 2 * (n_hi + 1) - 3:  # a tiled series: one tile size for both lengths
                rsv.rsv_set_schedule(ctx, nt, j, nt * j - 2 * (n_hi + 1) - 3)
            times = []
            try:
                for n_md in (n_lo, n_hi):
                    h = torch.tensor(s.h_true, device=dev)
                    th = torch.tensor(s.theta, dtype=torch.float64, device=dev)
                    n = 10 if prec == "mixed" else 2
                    rsv.rsv_hmc_chain(ctx, h, y, lr, th, n_md, 0.005, 2, prec=prec, seed=1)
                    torch.cuda.synchronize()
                    rsv.rsv_stats(ctx, reset=True)
                    rsv.rsv_timing(ctx, True)
                    rsv.rsv_hmc_chain(ctx, h, y, lr, th, n_md, 0.005, n, prec=prec, seed=2)
                    torch.cuda.synchronize()
                    rsv.rsv_timing(ctx, False)
                    _, nl, ms = rsv.rsv_stats(ctx, reset=True)
                    times.append(ms / 1e3 / max(nl, 1))
            finally:
                rsv.rsv_set_schedule(ctx)
            res["gpu_" + prec].append((times[1] - times[0]) / (n_hi - n_lo))
    return res


def table2_cpu(B_list):
    """Seconds per elementary step of the FP64 oracle's leapfrog on one host
    core, T = 512 B (part of the CPU baseline: the oracle as it stands)."""
    import oracle
    from paper_1603_08114_gb300 import synth
    out = []
    for B in B_list:
        T = 512 * B
        s = synth.rsv_series(T, synth.THETA_STD, seed=1)
        p0 = synth.standard_normals(T, 5)
        n_steps = max(2, min(200, int(2e6 // T)))
        t0 = time.perf_counter()
        oracle.leapfrog(s.h_true, p0, s.y, s.lnrv, s.theta, n_steps, 0.005)
        out.append((time.perf_counter() - t0) / n_steps)
    return out


def table2_summary(B_list, gpu, cpu):
    res = {"B": list(B_list), "T": [512 * b for b in B_list], **gpu}
    keys = ["gpu_mixed", "gpu_fp64"]
    if cpu is not None:
        res["cpu_oracle"] = cpu
        keys.append("cpu_oracle")
    fits = {k: dict(zip(("A", "C"), fit_linear(B_list, res[k]))) for k in keys}
    res.update({
        "unit": "seconds per elementary step (one leapfrog step over all T sites)",
        "fit": fits,
        "site_updates_per_s_at_largest_B": 512 * B_list[-1] / res["gpu_mixed"][-1],
        "paper": PAPER_TABLE2,
        "how": "GPU: trajectory time of a chain call (mixed: the persistent chain kernel; "
               "FP64: one k_traj_fp64 launch per trajectory) at n_md = 110 minus at n_md = 10 "
               "(one tiling, CUDA events) / 100; oracle: FP64 leapfrog in plain C on one "
               "host core; fitted f(B) = A + C B like the paper's Table 2"})
    if cpu is not None:
        res["gain_limit_mixed_vs_oracle"] = fits["cpu_oracle"]["C"] / fits["gpu_mixed"]["C"]
        res["gain_limit_fp64_vs_oracle"] = fits["cpu_oracle"]["C"] / fits["gpu_fp64"]["C"]
    return res


def run_table2(args):
    """The full B ladder of the elementary-step sweep (1 ... 2048)."""
    import torch

    from paper_1603_08114_gb300 import rsv, synth
    torch.cuda.set_device(0)
    ctx = rsv.Context(0)
    gpu = table2_gpu(ctx, rsv, synth, torch, TABLE2_B)
    cpu = table2_cpu(TABLE2_B)
    print(json.dumps({"table2": table2_summary(TABLE2_B, gpu, cpu)}))
    ctx.close()
    return 0


def run_profile_chain(args):
    """The headline's chain for a profiler: T = 2^20, a mass of the learned
    mass's shape (m ~ 30, fixed: no training), 78 x 0.035, theta sampled,
    every state recorded; one warm-up call, then one call of K trajectories
    (`ncu -k regex:k_chain_mixed -s 1 -c 1` takes that one).  With
    --profile-prec fp64: the FP64 arm's chain instead (identity mass, 100 x
    0.005, one k_traj_fp64 launch per trajectory)."""
    import torch

    from paper_1603_08114_gb300 import rsv, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = rsv.Context(0)
    K = int(args.profile_chain)
    # the same trajectory length at another step count (the leapfrog's share
    # of a launch: compare captures at two counts)
    n_md = int(args.profile_nmd)
    dtau = 0.035 * 78 / n_md
    fp64 = args.profile_prec == "fp64"
    if fp64:
        n_md, dtau = N_MD, DTAU
    if args.profile_tile:
        cs = rsv.rsv_chain_schedule(ctx, T_SITES, 78, "mixed", with_mass=True)
        rsv.rsv_set_schedule(ctx, cs["threads"], cs["sites_per_thread"], int(args.profile_tile))
    s = synth.rsv_series(T_SITES, synth.THETA_STD, seed=SEED_DATA)
    y, lnrv = torch.tensor(s.y, device=dev), torch.tensor(s.lnrv, device=dev)
    m = 30.0 + 3.0 * np.random.default_rng(3).random(T_SITES)
    minv = torch.tensor((1.0 / m).astype(np.float32), device=dev)
    rsv.rsv_reserve(ctx, T_SITES)
    h = torch.tensor(s.h_true, device=dev)
    th = torch.tensor(s.theta, dtype=torch.float64, device=dev)
    snaps = torch.empty(K, T_SITES, dtype=torch.float32, device=dev)
    thetas = torch.empty(K, 5, dtype=torch.float64, device=dev)
    acc = torch.empty(K, dtype=torch.int32, device=dev)
    for k in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rsv.rsv_hmc_chain(ctx, h, y, lnrv, th, n_md, dtau, K, prec="fp64" if fp64 else "mixed",
                          minv=None if fp64 else minv, seed=11, traj0=k * K, snaps=snaps, thin=1,
                          theta_out=thetas, accept_out=acc, update_theta=True)
        b.record()
        b.synchronize()
    rsv.rsv_sync_status(ctx)
    cs = rsv.rsv_chain_schedule(ctx, T_SITES, n_md, "fp64" if fp64 else "mixed",
                                with_mass=not fp64)
    print(json.dumps({"profile_chain": K, "prec": "fp64" if fp64 else "mixed", "n_md": n_md, "us_per_trajectory": 1e3 * a.elapsed_time(b) / K,
                      "accept_rate": float(acc.float().mean()), "schedule": cs}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mass-file", default=None,
                    help="npy of FP32 inverse masses for the headline arm")
    ap.add_argument("--only", default=None, choices=["mixed"],
                    help="run the headline arm only (profiling)")
    ap.add_argument("--traj-per-step", type=int, default=None,
                    help="trajectories per step (profiling; default 200)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-learned", action="store_true",
                    help="headline arm without the learned mass (profiling)")
    ap.add_argument("--n-snap", type=int, default=10000,
                    help="plain-sampler snapshots for the learned mass")
    ap.add_argument("--table2", action="store_true",
                    help="time per elementary step vs B (T = 512 B) like the paper's Table 2")
    ap.add_argument("--profile-chain", type=int, default=0,
                    help="run the headline chain twice with K trajectories (profiling)")
    ap.add_argument("--profile-nmd", type=int, default=78,
                    help="leapfrog steps per trajectory of --profile-chain (dtau 0.035 x 78 / n)")
    ap.add_argument("--profile-prec", default="mixed", choices=["mixed", "fp64"],
                    help="precision of --profile-chain's chain (fp64: the FP64 arm's)")
    ap.add_argument("--profile-tile", type=int, default=0,
                    help="owned sites per tile of --profile-chain, with the block shape of the "
                         "78-step chain (0: the planner's tiling)")
    args = ap.parse_args()
    if args.traj_per_step:
        global N_TRAJ
        N_TRAJ = int(args.traj_per_step)
    if args.warmup < 3:
        # the timing rules take at least 3 untimed steps; the line reports
        # the count that ran
        print(f"bench.py: --warmup {args.warmup} raised to 3 (at least 3 warm-up steps)",
              file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.table2:
        return run_table2(args)
    if args.profile_chain:
        return run_profile_chain(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
