"""The double-float exponential of the mixed path's energies and state
statistics (Sec. 3's return term (y^2/2) e^{-h}), against exp in FP64 over
-69 < t < 80 (below about -70 the small part of the result leaves FP32's
normal range and the relative error grows; the kernels' arguments are -h, a
few units at most), and its two-lane form against the scalar one bit for
bit.

Error bound: the reduction t = k ln2/32 + r leaves |r| <= ln2/64 ~ 0.0108; the
polynomial part q ~ r^2/2 <= 5.9e-5 is formed in FP32 (relative rounding
2^-24 a step, a few steps) and added to the double-float 1 + r, so the
result's relative error is below ~4 x 2^-24 x 5.9e-5 ~ 1.4e-11 plus the
double-float roundings (~2^-44) and the Taylor remainder r^6/720 < 2.2e-15.
The test takes 2e-11."""
import numpy as np
import pytest
import torch

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


def as_ff(t):
    """t rounded to a double-float exactly as the kernel holds it."""
    hi = t.astype(np.float32).astype(np.float64)
    lo = (t - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def test_ff_exp_against_fp64_exp(rsv, ctx):
    rng = np.random.default_rng(17)
    t = np.concatenate([
        rng.uniform(-69.0, 79.9, 200001),
        rng.uniform(-1.0, 1.0, 20000),
        rng.normal(0.0, 1e-3, 2000),
        # the reduction's boundaries: multiples of ln2/64 and their neighbours
        np.arange(-4000, 4001) * (np.log(2.0) / 64.0),
        np.nextafter(np.arange(-400, 401) * (np.log(2.0) / 64.0), np.inf),
        [0.0, -0.0, 1e-30, -1e-30, 79.9, -69.0],
    ])
    out, out2 = rsv.rsv_ff_exp(ctx, torch.tensor(t, dtype=torch.float64, device="cuda"))
    out, out2 = out.cpu().numpy(), out2.cpu().numpy()
    ref = np.exp(as_ff(t))
    rel = np.abs(out - ref) / ref
    assert rel.max() < 2e-11, (rel.max(), t[np.argmax(rel)])
    # the two-lane form is the scalar form lane by lane, bit for bit, while no
    # part of the result is subnormal (for t > -50: the kernels' arguments
    # are -h, a few units); below, the small part can reach FP32's subnormal
    # range, where the packed and the scalar FP32 instructions may differ in
    # it -- by less than the smallest normal float
    mid = t > -50.0
    diff = np.flatnonzero(mid & (out != out2))
    assert diff.size == 0, (diff.size, t[diff[:5]], out[diff[:5]], out2[diff[:5]])
    assert np.all(np.abs(out2 - out) <= np.finfo(np.float32).tiny), np.abs(out2 - out).max()
    rel2 = np.abs(out2 - ref) / ref
    assert rel2[mid].max() < 2e-11


def test_ff_exp_odd_count_and_empty(rsv, ctx):
    t = torch.tensor([0.5, -2.0, 3.25], dtype=torch.float64, device="cuda")
    out, out2 = rsv.rsv_ff_exp(ctx, t)
    ref = np.exp(as_ff(t.cpu().numpy()))
    assert np.all(np.abs(out.cpu().numpy() - ref) / ref < 2e-11)
    assert torch.equal(out, out2)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    a, b = rsv.rsv_ff_exp(ctx, e)
    assert a.numel() == 0 and b.numel() == 0


def test_fp64_table_exp_against_exp(rsv, ctx):
    """The FP64 path's table-driven exponential (Tang's method) within 2 ulp of
    exp over |t| < 700: the table's and the final fused step's roundings
    (0.5 ulp each), the reduction's tail and the degree-5 remainder (< 4e-17
    on |r| <= ln2/128) leave it within ~1.5 ulp of e^t, and numpy's exp is
    within 1 ulp of it."""
    rng = np.random.default_rng(23)
    l = np.log(2.0) / 64.0
    t = np.concatenate([
        rng.uniform(-700.0, 700.0, 200001),
        rng.uniform(-10.0, 10.0, 200000),
        np.arange(-20000, 20001) * l,
        np.nextafter(np.arange(-2000, 2001) * (l / 2), np.inf),
        [0.0, -0.0, 1e-300, -1e-300, 511.999, -511.999, 512.0, -512.0, 700.0, -700.0],
    ])
    out = rsv.rsv_fp64_exp(ctx, torch.tensor(t, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = np.exp(t)
    ulp = np.abs(out - ref) / np.spacing(ref)
    assert ulp.max() <= 2.0, (ulp.max(), t[np.argmax(ulp)])
    assert np.mean(ulp) < 0.5
