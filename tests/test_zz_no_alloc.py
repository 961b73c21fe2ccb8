"""rsv_action_noalloc: S(h) whose scratch is a fixed device array, for callers
that cannot allocate device memory (graph capture, a host-owned memory pool,
real-time loops).  Checked through the C ABI against rsv_action, twice in a row
(the second call reuses the array the first one left behind).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1603_08114_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_action_matches_rsv_action_twice():
    from paper_1603_08114_gb300 import rsv
    lib = rsv.lib()
    f = lib.rsv_action_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, rsv.Theta,
                  ctypes.c_void_p, ctypes.c_void_p]
    ctx = rsv.Context(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for T, seed in ((1 << 20, 1), (100003, 2)):   # two calls in a row, different sizes
        s = synth.rsv_series(T, synth.THETA_STD, seed=seed)
        h = torch.tensor(s.h0, device="cuda")
        y = torch.tensor(s.y, device="cuda")
        lr = torch.tensor(s.lnrv, device="cuda")
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = f(ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(y.data_ptr()),
               ctypes.c_void_p(lr.data_ptr()), T, rsv.theta(synth.THETA_STD),
               ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.rsv_last_error()
        ref = rsv.rsv_action(ctx, h, y, lr, synth.THETA_STD)
        torch.cuda.synchronize()
        a, b = out.item(), ref.item()
        assert np.isfinite(a)
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), (a, b)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1603_08114_gb300 import rsv
    lib = rsv.lib()
    f = lib.rsv_action_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, rsv.Theta,
                  ctypes.c_void_p, ctypes.c_void_p]
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # rejected before any launch: the arrays are never read
    st = f(p, p, p, 8388609, rsv.theta(synth.THETA_STD), p, None)
    assert st == 1  # RSV_EINVAL
    lib.rsv_last_error.restype = ctypes.c_char_p
    assert b"exceeds" in lib.rsv_last_error()
