"""FP64 CPU oracle for the RSV-model HMC volatility update (arXiv:1603.08114).

TEST INFRASTRUCTURE ONLY.  This package is the correctness reference the CUDA
library is checked against; the library never imports it.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

``rsv_oracle.c`` holds the arithmetic (plain FP64 loops, see its header for the
paper citations); this module compiles it with gcc and wraps it with ctypes.
``stats.py`` holds the MCMC-output estimators and ``mlp.py`` the FP64 reference
of the learned-mass network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_rsv.so")
_lock = threading.Lock()
_lib = None


class Theta(ctypes.Structure):
    """theta = (phi, mu, xi, sigma_eta^2, sigma_u^2), the parameters of eqs. (1)-(3),
    and rho = corr(eps_t, eta_t) of the RSV model with leverage (0 if not given)."""

    _fields_ = [("phi", ctypes.c_double), ("mu", ctypes.c_double), ("xi", ctypes.c_double),
                ("sig_eta2", ctypes.c_double), ("sig_u2", ctypes.c_double),
                ("rho", ctypes.c_double)]

    def as_tuple(self):
        return (self.phi, self.mu, self.xi, self.sig_eta2, self.sig_u2)

    def copy(self):
        return Theta(*self.as_tuple(), self.rho)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_site_action.restype = ctypes.c_double
            L.orc_site_action.argtypes = [_D, _D, _D, ctypes.c_long, Theta, ctypes.c_long]
            L.orc_action_sites.argtypes = [_D, _D, _D, ctypes.c_long, Theta, _D]
            L.orc_action.restype = ctypes.c_double
            L.orc_action.argtypes = [_D, _D, _D, ctypes.c_long, Theta]
            L.orc_force.argtypes = [_D, _D, _D, ctypes.c_long, Theta, _D]
            L.orc_leapfrog.argtypes = [_D, _D, _D, _D, ctypes.c_long, Theta, _D, ctypes.c_int,
                                       ctypes.c_double]
            L.orc_omelyan2.argtypes = [_D, _D, _D, _D, ctypes.c_long, Theta, _D, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double]
            L.orc_omelyan4.argtypes = [_D, _D, _D, _D, ctypes.c_long, Theta, _D, ctypes.c_int,
                                       ctypes.c_double]
            L.orc_delta_H.restype = ctypes.c_double
            L.orc_delta_H.argtypes = [_D, _D, _D, _D, _D, _D, ctypes.c_long, Theta, _D]
            L.orc_metropolis.restype = ctypes.c_int
            L.orc_metropolis.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_trajectory.restype = ctypes.c_int
            L.orc_trajectory.argtypes = [_D, _D, _D, _D, ctypes.c_long, Theta, _D, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, _D, ctypes.c_int,
                                         ctypes.c_double]
            L.orc_philox4x64_10.argtypes = [_U64, _U64, _U64]
            L.orc_u01.restype = ctypes.c_double
            L.orc_u01.argtypes = [ctypes.c_uint64, ctypes.c_int]
            L.orc_box_muller.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
            L.orc_draw_momenta.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_long, _D, ctypes.c_int, _D]
            L.orc_draw_log_u.restype = ctypes.c_double
            L.orc_draw_log_u.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            L.orc_gibbs_theta.restype = ctypes.c_int
            L.orc_gibbs_theta.argtypes = [_D, _D, ctypes.c_long, ctypes.POINTER(Theta),
                                          ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_int]
            L.orc_gibbs_theta_margin.restype = ctypes.c_int
            L.orc_gibbs_theta_margin.argtypes = [_D, _D, ctypes.c_long, ctypes.POINTER(Theta),
                                                 ctypes.c_uint64, ctypes.c_uint64,
                                                 ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                 _D]
            L.orc_chain.restype = ctypes.c_long
            L.orc_chain.argtypes = [_D, _D, _D, ctypes.c_long, ctypes.POINTER(Theta), _D,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_long, ctypes.c_int,
                                    ctypes.c_int, _D, _I, _D, _D, ctypes.c_long, ctypes.c_int,
                                    ctypes.c_double]
            _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def theta(th) -> Theta:
    if isinstance(th, Theta):
        return th
    return Theta(*[float(v) for v in th])


def action(h, y, lnrv, th) -> float:
    """S(h) = -ln f(h | theta, y, lnRV) up to constants (Sec. 3, model eqs. (1)-(3))."""
    h, y, lnrv = _f64(h), _f64(y), _f64(lnrv)
    return lib().orc_action(_d(h), _d(y), _d(lnrv), len(h), theta(th))


def action_sites(h, y, lnrv, th) -> np.ndarray:
    """Per-site split s_t of S(h) used for dH."""
    h, y, lnrv = _f64(h), _f64(y), _f64(lnrv)
    out = np.empty_like(h)
    lib().orc_action_sites(_d(h), _d(y), _d(lnrv), len(h), theta(th), _d(out))
    return out


def force(h, y, lnrv, th) -> np.ndarray:
    """dS/dh_t, the derivative in eq. (7)."""
    h, y, lnrv = _f64(h), _f64(y), _f64(lnrv)
    out = np.empty_like(h)
    lib().orc_force(_d(h), _d(y), _d(lnrv), len(h), theta(th), _d(out))
    return out


def leapfrog(h, p, y, lnrv, th, n_md, dtau, minv=None):
    """n_md leapfrog steps, eqs. (6)-(8); returns (h', p')."""
    h, p = _f64(h).copy(), _f64(p).copy()
    y, lnrv = _f64(y), _f64(lnrv)
    mv = None if minv is None else _f64(minv)
    lib().orc_leapfrog(_d(h), _d(p), _d(y), _d(lnrv), len(h), theta(th), _d(mv), int(n_md),
                       float(dtau))
    return h, p


def delta_H(h0, p0, h1, p1, y, lnrv, th, minv=None) -> float:
    """dH = H(p', h') - H(p, h) (Sec. 3)."""
    a = [_f64(v) for v in (h0, p0, h1, p1, y, lnrv)]
    mv = None if minv is None else _f64(minv)
    return lib().orc_delta_H(*[_d(v) for v in a], len(a[0]), theta(th), _d(mv))


def metropolis(dH, log_u) -> int:
    return lib().orc_metropolis(float(dH), float(log_u))


# lambda of the second-order minimum-norm integrator (Omelyan, Mryglod, Folk,
# Phys. Rev. E 65, 056706 (2002)): the root 1/2 - c/12 + 1/(6c),
# c = (2 sqrt(326) + 36)^(1/3), of its error-norm minimisation
LAMBDA_2MN = 0.19318332750378357

_INTEGRATORS = {"leapfrog": 0, "omelyan2": 1, "omelyan4": 2}

# The fourth-order minimum-norm scheme of Omelyan, Mryglod and Folk, Comput.
# Phys. Commun. 146, 188 (2002): drift coefficients (xi, chi, 1 - 2(chi + xi),
# chi, xi), kick coefficients ((1 - 2 lambda)/2, lambda, lambda, (1 - 2 lambda)/2).
PEFRL = {"xi": 0.1786178958448091, "lambda": -0.2123418310626054,
         "chi": -0.06626458266981849}


def omelyan2(h, p, y, lnrv, th, n_md, dtau, lam=LAMBDA_2MN, minv=None):
    """n_md steps of the minimum-norm integrator; returns (h', p')."""
    h, p = _f64(h).copy(), _f64(p).copy()
    y, lnrv = _f64(y), _f64(lnrv)
    mv = None if minv is None else _f64(minv)
    lib().orc_omelyan2(_d(h), _d(p), _d(y), _d(lnrv), len(h), theta(th), _d(mv), int(n_md),
                       float(dtau), float(lam))
    return h, p


def omelyan4(h, p, y, lnrv, th, n_md, dtau, minv=None):
    """n_md steps of the fourth-order scheme (four forces per step); returns (h', p')."""
    h, p = _f64(h).copy(), _f64(p).copy()
    y, lnrv = _f64(y), _f64(lnrv)
    mv = None if minv is None else _f64(minv)
    lib().orc_omelyan4(_d(h), _d(p), _d(y), _d(lnrv), len(h), theta(th), _d(mv), int(n_md),
                       float(dtau))
    return h, p


def trajectory(h, p, y, lnrv, th, n_md, dtau, log_u, minv=None, integrator="leapfrog",
               lam=LAMBDA_2MN):
    """One HMC trajectory; returns (h_new, p', dH, accept)."""
    h, p = _f64(h).copy(), _f64(p).copy()
    y, lnrv = _f64(y), _f64(lnrv)
    mv = None if minv is None else _f64(minv)
    dH = ctypes.c_double()
    acc = lib().orc_trajectory(_d(h), _d(p), _d(y), _d(lnrv), len(h), theta(th), _d(mv),
                               int(n_md), float(dtau), float(log_u), ctypes.byref(dH),
                               _INTEGRATORS[integrator], float(lam))
    return h, p, dH.value, acc


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib().orc_philox4x64_10(c.ctypes.data_as(_U64), k.ctypes.data_as(_U64),
                            out.ctypes.data_as(_U64))
    return out


def u01(w, bits=53) -> float:
    return lib().orc_u01(int(w), int(bits))


def box_muller(u1, u2):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().orc_box_muller(float(u1), float(u2), ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def draw_momenta(seed, series, traj, T, minv=None, bits=53) -> np.ndarray:
    p = np.empty(int(T), dtype=np.float64)
    mv = None if minv is None else _f64(minv)
    lib().orc_draw_momenta(int(seed), int(series), int(traj), int(T), _d(mv), int(bits), _d(p))
    return p


def draw_log_u(seed, series, traj) -> float:
    return lib().orc_draw_log_u(int(seed), int(series), int(traj))


def gibbs_theta(h, lnrv, th, seed, series, traj, mask=31):
    """One theta sweep (xi, s_u^2, mu, s_eta^2, phi; mask bits 0..4 select which);
    returns (theta', phi_accepted)."""
    h, lnrv = _f64(h), _f64(lnrv)
    t = theta(th).copy()
    acc = lib().orc_gibbs_theta(_d(h), _d(lnrv), len(h), ctypes.byref(t), int(seed), int(series),
                                int(traj), int(mask))
    if acc < 0:
        raise ValueError("the theta conditionals assume rho = 0")
    return t.as_tuple(), acc


def gibbs_theta_margin(h, lnrv, th, seed, series, traj, mask=31, bits=53):
    """gibbs_theta from uniforms of `bits` bits (53, or 23 as the FP32 sweep
    takes them), also returning the smallest distance of any accept/reject
    decision of the sweep from its boundary, |lhs - rhs| / (1 + |rhs|)."""
    h, lnrv = _f64(h), _f64(lnrv)
    t = theta(th).copy()
    m = ctypes.c_double()
    acc = lib().orc_gibbs_theta_margin(_d(h), _d(lnrv), len(h), ctypes.byref(t), int(seed),
                                       int(series), int(traj), int(mask), int(bits),
                                       ctypes.byref(m))
    if acc < 0:
        raise ValueError("the theta conditionals assume rho = 0")
    return t.as_tuple(), acc, m.value


def chain(h, y, lnrv, th, n_md, dtau, seed, n_traj, traj0=0, series=0, update_theta=False,
          bits=53, minv=None, thin=0, integrator="leapfrog", lam=LAMBDA_2MN):
    """n_traj trajectories with Philox draws; returns a dict of per-trajectory records."""
    h = _f64(h).copy()
    y, lnrv = _f64(y), _f64(lnrv)
    T = len(h)
    t = theta(th).copy()
    mv = None if minv is None else _f64(minv)
    dH = np.empty(n_traj)
    acc = np.empty(n_traj, dtype=np.int32)
    ths = np.empty((n_traj, 5))
    snaps = np.empty((n_traj // thin, T)) if thin else None
    n_acc = lib().orc_chain(_d(h), _d(y), _d(lnrv), T, ctypes.byref(t), _d(mv), int(n_md),
                            float(dtau), int(seed), int(series), int(traj0), int(n_traj),
                            int(bool(update_theta)), int(bits), _d(dH),
                            acc.ctypes.data_as(_I), _d(ths), _d(snaps), int(thin),
                            _INTEGRATORS[integrator], float(lam))
    if n_acc < 0:
        raise ValueError("the theta update assumes rho = 0")
    return dict(h=h, theta=t.as_tuple(), dH=dH, accept=acc, thetas=ths, snaps=snaps,
                n_accept=int(n_acc))
