"""Thin Python binding of librsv (include/rsv.h).

Argument marshalling only: every function checks tensor dtypes/devices, passes
raw device pointers and the current torch CUDA stream to the C entry point of
the same name, and turns a non-OK status into an exception.  There is no CPU
fallback: without librsv.so or a GPU the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

RSV_OK, RSV_EINVAL, RSV_ENOMEM, RSV_ECUDA, RSV_ENONFINITE, RSV_ETIMEOUT = range(6)
RSV_FP64, RSV_MIXED = 0, 1
_STATUS = {0: "RSV_OK", 1: "RSV_EINVAL", 2: "RSV_ENOMEM", 3: "RSV_ECUDA", 4: "RSV_ENONFINITE",
           5: "RSV_ETIMEOUT"}


class RSVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Theta(ctypes.Structure):
    """rsv_theta: (phi, mu, xi, sigma_eta^2, sigma_u^2)."""
    _fields_ = [("phi", ctypes.c_double), ("mu", ctypes.c_double), ("xi", ctypes.c_double),
                ("sig_eta2", ctypes.c_double), ("sig_u2", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_INT = ctypes.c_int


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load librsv.so (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: the CUDA library is not built "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ctypes.CDLL(path)
        L.rsv_last_error.restype = ctypes.c_char_p
        L.rsv_abi_version.restype = _INT
        L.rsv_create.argtypes = [ctypes.POINTER(_P), _INT]
        L.rsv_destroy.argtypes = [_P]
        L.rsv_destroy.restype = None
        L.rsv_reserve.argtypes = [_P, _I64, _I64]
        L.rsv_sync_status.argtypes = [_P, _P]
        L.rsv_set_schedule.argtypes = [_P, _INT, _INT, _I64]
        L.rsv_set_integrator.argtypes = [_P, _INT, ctypes.c_double]
        L.rsv_set_leverage.argtypes = [_P, ctypes.c_double]
        L.rsv_set_persistent.argtypes = [_P, _INT]
        L.rsv_set_wait_limit.argtypes = [_P, _I64]
        L.rsv_chain_schedule.argtypes = [_P, _I64, _INT, _INT, _INT, ctypes.POINTER(_INT),
                                         ctypes.POINTER(_INT), ctypes.POINTER(_I64),
                                         ctypes.POINTER(_INT)]
        L.rsv_action.argtypes = [_P, _P, _P, _P, _I64, Theta, _P, _P]
        L.rsv_force.argtypes = [_P, _P, _P, _P, _I64, Theta, _P, _P]
        L.rsv_hmc_trajectory.argtypes = [_P, _P, _P, _P, _P, _I64, Theta, _P, _INT,
                                         ctypes.c_double, _INT, _U64, _U64, _P, _P, _P, _P]
        L.rsv_hmc_chain.argtypes = [_P, _P, _P, _P, _I64, _P, _P, _INT, ctypes.c_double, _INT,
                                    _U64, _U64, _I64, _INT, _P, _P, _P, _P, _I64, _INT, _P, _P]
        L.rsv_draw_momenta.argtypes = [_P, _U64, _U64, _U64, _I64, _P, _INT, _P, _P]
        L.rsv_ess.argtypes = [_P, _P, _I64, _I64, _P, _P]
        L.rsv_gibbs_theta.argtypes = [_P, _P, _P, _I64, _P, _U64, _U64, _U64, _INT, _INT, _P, _P]
        L.rsv_plan_create.argtypes = [_P, _P, _I64, _INT, _INT, _INT, ctypes.POINTER(_P)]
        L.rsv_plan_destroy.argtypes = [_P]
        L.rsv_plan_destroy.restype = None
        L.rsv_plan_info.argtypes = [_P] + [ctypes.POINTER(_INT)] * 5
        L.rsv_hmc_batched.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_double, _U64,
                                      _U64, _I64, _P, _P, _P, _P]
        L.rsv_timing.argtypes = [_P, _INT]
        L.rsv_pipe_probe.argtypes = [_P, _INT, _I64, ctypes.POINTER(ctypes.c_double), _P]
        L.rsv_ff_exp.argtypes = [_P, _P, _P, _P, _I64, _P]
        L.rsv_fp64_exp.argtypes = [_P, _P, _P, _I64, _P]
        L.rsv_stats.argtypes = [_P, _INT, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                ctypes.POINTER(ctypes.c_double)]
        for name in ("rsv_create", "rsv_reserve", "rsv_sync_status", "rsv_set_schedule",
                     "rsv_set_integrator", "rsv_set_leverage", "rsv_action", "rsv_force",
                     "rsv_hmc_trajectory", "rsv_hmc_chain", "rsv_draw_momenta", "rsv_ess",
                     "rsv_timing", "rsv_stats", "rsv_gibbs_theta", "rsv_plan_create",
                     "rsv_plan_info", "rsv_hmc_batched", "rsv_pipe_probe", "rsv_set_persistent",
                     "rsv_set_wait_limit", "rsv_chain_schedule", "rsv_ff_exp", "rsv_fp64_exp"):
            getattr(L, name).restype = _INT
        _lib = L
    return _lib


def _check(st: int):
    if st != RSV_OK:
        raise RSVError(st, lib().rsv_last_error().decode(errors="replace"))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype, n=None, name="array"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return ctypes.c_void_p(t.data_ptr())


def theta(th) -> Theta:
    if isinstance(th, Theta):
        return th
    return Theta(*[float(v) for v in th])


class Context:
    """An rsv_ctx bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        h = _P()
        _check(lib().rsv_create(ctypes.byref(h), int(device)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().rsv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsv_reserve(ctx: Context, max_T: int, max_series: int = 0):
    _check(lib().rsv_reserve(ctx.handle, int(max_T), int(max_series)))


RSV_LEAPFROG, RSV_OMELYAN2 = 0, 1
RSV_OMELYAN2_LAMBDA = 0.19318332750378357
RSV_OMELYAN4 = 2


def rsv_set_integrator(ctx: Context, kind="leapfrog", lam: float = 0.0):
    """Integrator of later trajectories and plans: "leapfrog", "omelyan2"
    (lam <= 0: the minimum-norm value) or "omelyan4" (lam ignored)."""
    k = {"leapfrog": RSV_LEAPFROG, "omelyan2": RSV_OMELYAN2,
         "omelyan4": RSV_OMELYAN4}.get(kind, kind)
    _check(lib().rsv_set_integrator(ctx.handle, int(k), float(lam)))


def rsv_set_persistent(ctx: Context, enable: bool = True):
    """Run mixed single-series chains as one persistent launch (default) or
    one trajectory kernel per trajectory."""
    _check(lib().rsv_set_persistent(ctx.handle, int(bool(enable))))


def rsv_set_wait_limit(ctx: Context, cycles: int = 0):
    """Clock cycles a device-side wait may spin before RSV_ETIMEOUT (0: default)."""
    _check(lib().rsv_set_wait_limit(ctx.handle, int(cycles)))


def rsv_chain_schedule(ctx: Context, T: int, n_md: int, prec="mixed", with_mass=False):
    """The block shape of an rsv_hmc_chain call and whether it runs persistent."""
    nt, j, tile, pers = _INT(), _INT(), _I64(), _INT()
    _check(lib().rsv_chain_schedule(ctx.handle, int(T), int(n_md), _prec(prec),
                                    int(bool(with_mass)), ctypes.byref(nt), ctypes.byref(j),
                                    ctypes.byref(tile), ctypes.byref(pers)))
    return {"threads": nt.value, "sites_per_thread": j.value, "tile": tile.value,
            "persistent": bool(pers.value)}


def rsv_set_leverage(ctx: Context, rho: float = 0.0):
    """Leverage corr(eps_t, eta_t) = rho of the RSV model for later calls and
    plans of this context (0: eqs. (1)-(3))."""
    _check(lib().rsv_set_leverage(ctx.handle, float(rho)))


def rsv_set_schedule(ctx: Context, threads: int = 0, sites_per_thread: int = 0, tile: int = 0):
    _check(lib().rsv_set_schedule(ctx.handle, int(threads), int(sites_per_thread), int(tile)))


def rsv_sync_status(ctx: Context, allow_nonfinite: bool = False) -> int:
    """Synchronise the current stream and clear the device status word; raise on
    a device-side condition.  With allow_nonfinite, RSV_ENONFINITE (a trajectory
    whose dH was not finite, rejected by the Metropolis test) is returned
    instead of raised."""
    st = lib().rsv_sync_status(ctx.handle, _stream())
    if allow_nonfinite and st == RSV_ENONFINITE:
        return st
    _check(st)
    return st


def rsv_action(ctx: Context, h, y, lnrv, th, S_out=None):
    T = h.numel()
    if S_out is None:
        S_out = torch.empty(1, dtype=torch.float64, device=h.device)
    _check(lib().rsv_action(ctx.handle, _ptr(h, torch.float64, T, "h"),
                            _ptr(y, torch.float64, T, "y"), _ptr(lnrv, torch.float64, T, "lnrv"),
                            T, theta(th), _ptr(S_out, torch.float64, 1, "S_out"), _stream()))
    return S_out


def rsv_force(ctx: Context, h, y, lnrv, th, F_out=None):
    T = h.numel()
    if F_out is None:
        F_out = torch.empty_like(h)
    _check(lib().rsv_force(ctx.handle, _ptr(h, torch.float64, T, "h"),
                           _ptr(y, torch.float64, T, "y"), _ptr(lnrv, torch.float64, T, "lnrv"),
                           T, theta(th), _ptr(F_out, torch.float64, T, "F_out"), _stream()))
    return F_out


def _prec(prec) -> int:
    if prec in (RSV_FP64, "fp64", "f64"):
        return RSV_FP64
    if prec in (RSV_MIXED, "mixed"):
        return RSV_MIXED
    raise ValueError(f"unknown precision {prec!r}")


def rsv_hmc_trajectory(ctx: Context, h, p, y, lnrv, th, n_md: int, dtau: float, prec="fp64",
                       minv=None, seed: int = 0, traj: int = 0, log_u=None, dH_out=None,
                       accept_out=None):
    """One trajectory in place on h (and p if given); returns (dH, accept) device tensors."""
    T = h.numel()
    dev = h.device
    if dH_out is None:
        dH_out = torch.empty(1, dtype=torch.float64, device=dev)
    if accept_out is None:
        accept_out = torch.empty(1, dtype=torch.int32, device=dev)
    _check(lib().rsv_hmc_trajectory(
        ctx.handle, _ptr(h, torch.float64, T, "h"), _ptr(p, torch.float64, T, "p"),
        _ptr(y, torch.float64, T, "y"), _ptr(lnrv, torch.float64, T, "lnrv"), T, theta(th),
        _ptr(minv, torch.float32, T, "minv"), int(n_md), float(dtau), _prec(prec), int(seed),
        int(traj), _ptr(log_u, torch.float64, 1, "log_u"), _ptr(dH_out, torch.float64, 1, "dH"),
        _ptr(accept_out, torch.int32, 1, "accept"), _stream()))
    return dH_out, accept_out


def rsv_hmc_chain(ctx: Context, h, y, lnrv, theta_dev, n_md: int, dtau: float, n_traj: int,
                  prec="fp64", minv=None, seed: int = 0, traj0: int = 0, update_theta=False,
                  dH_out=None, accept_out=None, theta_out=None, snaps=None, thin: int = 1,
                  fallback_window: int = 0, mass_used_out=None):
    """n_traj trajectories in place on h and theta_dev (device FP64 [5])."""
    T = h.numel()
    _check(lib().rsv_hmc_chain(
        ctx.handle, _ptr(h, torch.float64, T, "h"), _ptr(y, torch.float64, T, "y"),
        _ptr(lnrv, torch.float64, T, "lnrv"), T, _ptr(theta_dev, torch.float64, 5, "theta"),
        _ptr(minv, torch.float32, T, "minv"), int(n_md), float(dtau), _prec(prec), int(seed),
        int(traj0), int(n_traj), int(bool(update_theta)),
        _ptr(dH_out, torch.float64, n_traj, "dH_out"),
        _ptr(accept_out, torch.int32, n_traj, "accept_out"),
        _ptr(theta_out, torch.float64, 5 * n_traj, "theta_out"),
        _ptr(snaps, torch.float32, (n_traj // max(thin, 1)) * T if snaps is not None else None,
             "snaps"),
        int(thin), int(fallback_window), _ptr(mass_used_out, torch.int32, 1, "mass_used_out"),
        _stream()))


def rsv_draw_momenta(ctx: Context, seed: int, series: int, traj: int, T: int, minv=None,
                     bits: int = 53, device="cuda"):
    p = torch.empty(int(T), dtype=torch.float64, device=device)
    _check(lib().rsv_draw_momenta(ctx.handle, int(seed), int(series), int(traj), int(T),
                                  _ptr(minv, torch.float32, T, "minv"), int(bits),
                                  _ptr(p, torch.float64, T, "p"), _stream()))
    return p


def rsv_ess(ctx: Context, x):
    """ESS of every column of x, a [n, T] FP32 CUDA tensor of chain samples."""
    n, T = x.shape
    out = torch.empty(T, dtype=torch.float32, device=x.device)
    _check(lib().rsv_ess(ctx.handle, _ptr(x, torch.float32, n * T, "x"), int(n), int(T),
                         _ptr(out, torch.float32, T, "ess_out"), _stream()))
    return out


def rsv_ff_exp(ctx: Context, t):
    """The mixed path's double-float exponential at the FP64 CUDA tensor t
    (each argument rounded to a double-float): (scalar form, two-lane form)."""
    n = t.numel()
    out = torch.empty(n, dtype=torch.float64, device=t.device)
    out2 = torch.empty(n, dtype=torch.float64, device=t.device)
    _check(lib().rsv_ff_exp(ctx.handle, _ptr(t, torch.float64, n, "t"),
                            _ptr(out, torch.float64, n, "out"), _ptr(out2, torch.float64, n, "out2"),
                            int(n), _stream()))
    return out, out2


def rsv_fp64_exp(ctx: Context, t):
    """The FP64 path's table-driven exponential at the FP64 CUDA tensor t."""
    n = t.numel()
    out = torch.empty(n, dtype=torch.float64, device=t.device)
    _check(lib().rsv_fp64_exp(ctx.handle, _ptr(t, torch.float64, n, "t"),
                              _ptr(out, torch.float64, n, "out"), int(n), _stream()))
    return out


PROBE_KINDS = {"ffma": 0, "ffma2": 1, "ex2": 2, "lds": 3, "dfma": 4}


def rsv_pipe_probe(ctx: Context, kind: str, iters: int) -> float:
    """Launch one pipe-probe kernel on the current stream; returns the number
    of operations it performs (FMAs, ex2, or bytes for "lds")."""
    ops = ctypes.c_double()
    _check(lib().rsv_pipe_probe(ctx.handle, PROBE_KINDS[kind], int(iters), ctypes.byref(ops),
                                _stream()))
    return ops.value


def rsv_timing(ctx: Context, enable: bool = True):
    _check(lib().rsv_timing(ctx.handle, int(bool(enable))))


def rsv_stats(ctx: Context, reset: bool = True):
    """(launches, trajectory launches, trajectory-kernel ms) since the last reset."""
    a, b, ms = _I64(), _I64(), ctypes.c_double()
    _check(lib().rsv_stats(ctx.handle, int(bool(reset)), ctypes.byref(a), ctypes.byref(b),
                           ctypes.byref(ms)))
    return a.value, b.value, ms.value


def rsv_gibbs_theta(ctx: Context, h, lnrv, theta_dev, seed: int, series: int = 0, traj: int = 0,
                    mask: int = 31, phi_acc_out=None, prec: str = "fp64"):
    """One theta Gibbs sweep in place on theta_dev (device FP64 [5]) given h."""
    T = h.numel()
    _check(lib().rsv_gibbs_theta(ctx.handle, _ptr(h, torch.float64, T, "h"),
                                 _ptr(lnrv, torch.float64, T, "lnrv"), T,
                                 _ptr(theta_dev, torch.float64, 5, "theta"), int(seed),
                                 int(series), int(traj), int(mask), _prec(prec),
                                 _ptr(phi_acc_out, torch.int32, 1, "phi_acc_out"), _stream()))


class Plan:
    """An rsv_plan: n independent series packed end to end (offsets [n+1])."""

    def __init__(self, ctx: Context, offsets, n_md: int, prec="mixed", with_mass=False):
        import numpy as np
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.n_series = len(off) - 1
        self.total = int(off[-1])
        self.ctx = ctx
        self.prec = _prec(prec)
        h = _P()
        _check(lib().rsv_plan_create(ctx.handle, off.ctypes.data_as(_P), self.n_series, int(n_md),
                                     self.prec, int(bool(with_mass)), ctypes.byref(h)))
        self.handle = h

    def info(self):
        v = [_INT() for _ in range(5)]
        _check(lib().rsv_plan_info(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(("threads", "sites_per_thread", "bins", "grid", "split_series"),
                        [x.value for x in v]))

    def close(self):
        if getattr(self, "handle", None):
            lib().rsv_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsv_plan_create(ctx: Context, offsets, n_md: int, prec="mixed", with_mass=False) -> Plan:
    return Plan(ctx, offsets, n_md, prec, with_mass)


def rsv_hmc_batched(ctx: Context, plan: Plan, h, y, lnrv, theta_dev, dtau: float, p=None,
                    minv=None, seed: int = 0, traj0: int = 0, n_traj: int = 1, log_u=None,
                    dH_out=None, accept_out=None):
    """n_traj trajectories of every series of the plan, in place on h (packed FP64)."""
    N, n = plan.total, plan.n_series
    _check(lib().rsv_hmc_batched(
        ctx.handle, plan.handle, _ptr(h, torch.float64, N, "h"), _ptr(p, torch.float64, N, "p"),
        _ptr(y, torch.float64, N, "y"), _ptr(lnrv, torch.float64, N, "lnrv"),
        _ptr(theta_dev, torch.float64, 5 * n, "theta"), _ptr(minv, torch.float32, N, "minv"),
        float(dtau), int(seed), int(traj0), int(n_traj), _ptr(log_u, torch.float64, n, "log_u"),
        _ptr(dH_out, torch.float64, n * n_traj, "dH_out"),
        _ptr(accept_out, torch.int32, n * n_traj, "accept_out"), _stream()))


RSV_MLP_NPARAM = 1761


def _mlp_lib():
    L = lib()
    if not getattr(L, "_mlp_ready", False):
        L.rsv_welford_update.argtypes = [_P, _P, _I64, _I64, _I64, _P, _P, _P]
        L.rsv_welford_target.argtypes = [_P, _P, _P, _I64, _I64, _P, _P, _P, _P]
        L.rsv_mass_features.argtypes = [_P, _P, _P, _P, _I64, Theta, _P, _P, _P]
        L.rsv_mlp_grad.argtypes = [_P, _P, _P, _I64, _P, _P, _U64, _U64, _INT, _P, _P, _P]
        L.rsv_mlp_train.argtypes = [_P, _P, _P, _I64, _P, _P, _P, _P, _I64, _INT, _INT, _U64,
                                    ctypes.c_float, _P, _P]
        L.rsv_mlp_mass.argtypes = [_P, _P, _I64, _P, _P, _P, _P, Theta, _P, _P, _P]
        for n in ("rsv_welford_update", "rsv_welford_target", "rsv_mass_features",
                  "rsv_mlp_grad", "rsv_mlp_train", "rsv_mlp_mass"):
            getattr(L, n).restype = _INT
        L._mlp_ready = True
    return L


def rsv_welford_update(ctx: Context, x, count: int, mean, m2):
    """Fold the rows of x ([n, T] FP32) into running (count, mean, M2) FP64."""
    n, T = x.shape
    _check(_mlp_lib().rsv_welford_update(ctx.handle, _ptr(x, torch.float32, n * T, "x"), n, T,
                                         int(count), _ptr(mean, torch.float64, T, "mean"),
                                         _ptr(m2, torch.float64, T, "m2"), _stream()))
    return count + n


def rsv_welford_target(ctx: Context, mean, m2, count: int, hbar_out=None, target_out=None,
                       log_scale_out=None):
    T = mean.numel()
    if target_out is None:
        target_out = torch.empty(T, dtype=torch.float32, device=mean.device)
    _check(_mlp_lib().rsv_welford_target(ctx.handle, _ptr(mean, torch.float64, T, "mean"),
                                         _ptr(m2, torch.float64, T, "m2"), T, int(count),
                                         _ptr(hbar_out, torch.float64, T, "hbar_out"),
                                         _ptr(target_out, torch.float32, T, "target_out"),
                                         _ptr(log_scale_out, torch.float32, 1, "log_scale_out"),
                                         _stream()))
    return target_out


def rsv_mass_features(ctx: Context, y, lnrv, hbar, th):
    T = y.numel()
    feat = torch.empty(T, 20, dtype=torch.float32, device=y.device)
    stats = torch.empty(40, dtype=torch.float32, device=y.device)
    _check(_mlp_lib().rsv_mass_features(ctx.handle, _ptr(y, torch.float64, T, "y"),
                                        _ptr(lnrv, torch.float64, T, "lnrv"),
                                        _ptr(hbar, torch.float64, T, "hbar"), T, theta(th),
                                        _ptr(feat, torch.float32, 20 * T, "feat"),
                                        _ptr(stats, torch.float32, 40, "stats"), _stream()))
    return feat, stats


def rsv_mlp_grad(ctx: Context, feat, target, params, seed: int, step: int, batch: int,
                 log_scale=None):
    T = target.numel()
    g = torch.empty(RSV_MLP_NPARAM, dtype=torch.float32, device=feat.device)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    _check(_mlp_lib().rsv_mlp_grad(ctx.handle, _ptr(feat, torch.float32, 20 * T, "feat"),
                                   _ptr(target, torch.float32, T, "target"), T,
                                   _ptr(params, torch.float32, RSV_MLP_NPARAM, "params"),
                                   _ptr(log_scale, torch.float32, 1, "log_scale"),
                                   int(seed), int(step), int(batch),
                                   _ptr(g, torch.float32, RSV_MLP_NPARAM, "grad"),
                                   _ptr(loss, torch.float32, 1, "loss"), _stream()))
    return g, loss


def rsv_mlp_train(ctx: Context, feat, target, params, adam_m, adam_v, step0: int, n_steps: int,
                  batch: int, seed: int, lr: float = 1e-3, loss_out=None, log_scale=None):
    T = target.numel()
    _check(_mlp_lib().rsv_mlp_train(ctx.handle, _ptr(feat, torch.float32, 20 * T, "feat"),
                                    _ptr(target, torch.float32, T, "target"), T,
                                    _ptr(params, torch.float32, RSV_MLP_NPARAM, "params"),
                                    _ptr(log_scale, torch.float32, 1, "log_scale"),
                                    _ptr(adam_m, torch.float32, RSV_MLP_NPARAM, "adam_m"),
                                    _ptr(adam_v, torch.float32, RSV_MLP_NPARAM, "adam_v"),
                                    int(step0), int(n_steps), int(batch), int(seed), float(lr),
                                    _ptr(loss_out, torch.float32, n_steps, "loss_out"),
                                    _stream()))


def rsv_mlp_mass(ctx: Context, feat, params, y, hbar, th, m_out=None, log_scale=None):
    T = feat.shape[0]
    minv = torch.empty(T, dtype=torch.float32, device=feat.device)
    _check(_mlp_lib().rsv_mlp_mass(ctx.handle, _ptr(feat, torch.float32, 20 * T, "feat"), T,
                                   _ptr(params, torch.float32, RSV_MLP_NPARAM, "params"),
                                   _ptr(log_scale, torch.float32, 1, "log_scale"),
                                   _ptr(y, torch.float64, T, "y"),
                                   _ptr(hbar, torch.float64, T, "hbar"), theta(th),
                                   _ptr(minv, torch.float32, T, "minv"),
                                   _ptr(m_out, torch.float32, T, "m_out"), _stream()))
    return minv
