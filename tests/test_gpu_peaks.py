"""The pipe-probe kernels (rsv_pipe_probe) run and give rates in the range the
GB300's unit counts allow: 152 SMs x 128 FP32 lanes, 16 special-function
lanes and 128 bytes of shared memory per clock, at 1.0-2.1 GHz."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsv():
    from paper_1603_08114_gb300 import rsv as r
    return r


def rate(rsv, ctx, kind, iters):
    rsv.rsv_pipe_probe(ctx, kind, iters)  # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ops = rsv.rsv_pipe_probe(ctx, kind, iters)
    b.record()
    b.synchronize()
    return ops / (a.elapsed_time(b) * 1e-3)


@pytest.mark.parametrize("kind,lo,hi", [
    ("ffma", 0.3 * 152 * 128 * 1.0e9, 1.05 * 152 * 128 * 2.07e9),
    ("ffma2", 0.3 * 152 * 128 * 1.0e9, 2.1 * 152 * 128 * 2.07e9),
    ("ex2", 0.3 * 152 * 16 * 1.0e9, 2.1 * 152 * 16 * 2.07e9),
    ("lds", 0.3 * 152 * 128 * 1.0e9, 1.05 * 152 * 128 * 2.07e9),
    ("dfma", 1e9, 152 * 64 * 2.07e9),
])
def test_probe_rates_are_plausible(rsv, kind, lo, hi):
    ctx = rsv.Context(0)
    try:
        r = rate(rsv, ctx, kind, 200 if kind != "dfma" else 20)
        rsv.rsv_sync_status(ctx)
    finally:
        ctx.close()
    assert lo < r < hi, (kind, r)


def test_probe_rejects_bad_arguments(rsv):
    import ctypes
    ctx = rsv.Context(0)
    ops = ctypes.c_double()
    try:
        # checked before any launch
        assert rsv.lib().rsv_pipe_probe(ctx.handle, 9, 10, ctypes.byref(ops), None) == 1
        assert rsv.lib().rsv_pipe_probe(ctx.handle, 0, 0, ctypes.byref(ops), None) == 1
        assert rsv.lib().rsv_pipe_probe(ctx.handle, 0, 10, None, None) == 1
    finally:
        ctx.close()
