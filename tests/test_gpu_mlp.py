"""Learned mass on the GPU against the FP64 reference (oracle/mlp.py): moments,
features, forward, gradients, Adam; and what the trained mass gains."""
import numpy as np
import pytest
import torch

from oracle import mlp, stats
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


def flat(P):
    return np.concatenate([P["W1"].ravel(), P["b1"], P["W2"].ravel(), P["b2"], P["W3"],
                           P["b3"]]).astype(np.float32)


def unflat(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0
    P = {}
    for k, shape in (("W1", (32, 20)), ("b1", (32,)), ("W2", (32, 32)), ("b2", (32,)),
                     ("W3", (32,)), ("b3", (1,))):
        n = int(np.prod(shape))
        P[k] = v[o:o + n].reshape(shape)
        o += n
    return P


def test_welford_matches_two_pass(rsv, ctx):
    rng = np.random.default_rng(0)
    n1, n2, T = 37, 50, 3001
    X = (rng.standard_normal((n1 + n2, T)) * rng.uniform(0.1, 2, T) + rng.uniform(-1, 1, T))
    X = X.astype(np.float32)
    mean = torch.zeros(T, dtype=torch.float64, device="cuda")
    m2 = torch.zeros_like(mean)
    c = rsv.rsv_welford_update(ctx, dev(X[:n1], torch.float32), 0, mean, m2)
    c = rsv.rsv_welford_update(ctx, dev(X[n1:], torch.float32), c, mean, m2)
    m, v = mlp.welford_reference(X)
    assert np.allclose(mean.cpu().numpy(), m, rtol=0, atol=1e-12)
    assert np.allclose(m2.cpu().numpy() / (c - 1), v, rtol=1e-11)
    hbar = torch.empty_like(mean)
    ls = torch.empty(1, dtype=torch.float32, device="cuda")
    tgt = rsv.rsv_welford_target(ctx, mean, m2, c, hbar_out=hbar, log_scale_out=ls).cpu().numpy()
    assert np.allclose(tgt, np.log(1 / v), rtol=0, atol=1e-5)
    assert abs(ls.item() - np.log(1 / v).mean()) < 1e-5
    assert np.array_equal(hbar.cpu().numpy(), mean.cpu().numpy())


def test_features_match_reference(rsv, ctx):
    T = 5003
    s = synth.rsv_series(T, TH, seed=4)
    hbar = s.h_true + 0.1 * np.cos(np.arange(T))
    F, st = rsv.rsv_mass_features(ctx, dev(s.y), dev(s.lnrv), dev(hbar), TH)
    ref, m, inv = mlp.standardize(mlp.features_raw(s.y, s.lnrv, hbar, s.theta))
    assert np.max(np.abs(F.cpu().numpy() - ref)) < 2e-5
    assert np.allclose(st.cpu().numpy()[:20], m, rtol=1e-6, atol=1e-6)


@pytest.fixture(scope="module")
def problem(rsv, ctx):
    T = 20000
    s = synth.rsv_series(T, TH, seed=5)
    hbar = s.h_true
    F, _ = rsv.rsv_mass_features(ctx, dev(s.y), dev(s.lnrv), dev(hbar), TH)
    target = (-np.log(0.02 + 0.01 * np.cos(np.arange(T) * 0.01) ** 2)).astype(np.float32)
    P = mlp.init_params(2)
    log_s = float(np.float32(target.mean()))
    return dict(T=T, F=F, Fnp=F.cpu().numpy().astype(np.float64), target=dev(target, torch.float32),
                target_np=target.astype(np.float64), P=P, series=s, log_s=log_s,
                log_s_dev=dev([log_s], torch.float32))


@pytest.mark.parametrize("scaled", [False, True])
def test_forward_matches_reference(rsv, ctx, problem, scaled):
    params = dev(flat(problem["P"]), torch.float32)
    m_gpu = torch.empty(problem["T"], dtype=torch.float32, device="cuda")
    s = problem["series"]
    ls = problem["log_s"] if scaled else 0.0
    minv = rsv.rsv_mlp_mass(ctx, problem["F"], params, dev(s.y), dev(s.h_true), TH, m_out=m_gpu,
                            log_scale=problem["log_s_dev"] if scaled else None).cpu().numpy()
    ref = mlp.forward(unflat(flat(problem["P"])), problem["Fnp"], bf=True, log_s=ls)["m"]
    lo, hi = mlp.mass_bounds(s.y, s.h_true, TH)
    ref = np.clip(ref, lo, hi)
    rel = np.abs(m_gpu.cpu().numpy() - ref) / ref
    assert np.median(rel) < 1e-5 and np.max(rel) < 5e-3
    assert np.allclose(minv, 1 / m_gpu.cpu().numpy(), rtol=1e-6)


@pytest.mark.parametrize("scaled", [False, True])
def test_forward_against_fp64_network_within_bf16_bound(rsv, ctx, problem, scaled):
    """The GPU network (BF16 operands, FP32 accumulation) against the plain
    FP64 network, within a tolerance derived from BF16 rounding.  Rounding
    to nearest BF16 (8 significant bits) moves each rounded operand x -- the
    features, W1, the hidden activations a1 and W2 -- to x (1 + e), |e| <= 2^-8;
    taken as independent with variance (2^-8)^2 / 3 (probabilistic rounding
    error analysis, Higham and Mary, SIAM J. Sci. Comput. 41 (2019) A2815),
    the first-order error of ln m at a site has the standard deviation
      sigma = 2^-8 / sqrt(3) * || x * d(ln m)/dx ||_2  over the rounded operands,
    the gradient taken through the FP64 network.  Every site must lie within
    6 sigma (+ 1e-5 for FP32 accumulation and the FP32 tanh, exp and log1p),
    and the errors must look like BF16 rounding: RMS of err / sigma <= 1.5
    and visibly above FP32 level."""
    P = unflat(flat(problem["P"]))   # the FP32 parameters the GPU holds
    params = dev(flat(problem["P"]), torch.float32)
    m_gpu = torch.empty(problem["T"], dtype=torch.float32, device="cuda")
    s = problem["series"]
    ls = problem["log_s"] if scaled else 0.0
    rsv.rsv_mlp_mass(ctx, problem["F"], params, dev(s.y), dev(s.h_true), TH, m_out=m_gpu,
                     log_scale=problem["log_s_dev"] if scaled else None)
    F = problem["Fnp"]
    ref = mlp.forward(P, F, bf=False, log_s=ls)
    a1, a2 = ref["a1"], ref["a2"]
    # d ln m / d z3, then back through the layers
    d3 = (1.0 / (1.0 + np.exp(-ref["z3"]))) / ref["u"]
    d2 = d3[:, None] * P["W3"][None, :] * (1.0 - a2 ** 2)        # d/dz2_k
    e1 = d2 @ P["W2"]                                             # d/d(rounded a1)_j
    d1 = e1 * (1.0 - a1 ** 2)                                     # d/dz1_j
    g2 = (e1 * a1) ** 2                                           # a1 rounding
    g2 += (d2 ** 2) @ (P["W2"] ** 2) * a1 ** 2                    # W2 rounding
    g2 = g2.sum(1)
    g2 += ((d1 @ P["W1"]) * F) ** 2 @ np.ones(F.shape[1])         # feature rounding
    g2 += ((d1 ** 2) @ (P["W1"] ** 2) * F ** 2).sum(1)            # W1 rounding
    sigma = 2.0 ** -8 / np.sqrt(3.0) * np.sqrt(g2)
    lo, hi = mlp.mass_bounds(s.y, s.h_true, TH)
    m_ref = np.clip(ref["m"], lo, hi)   # the clamp is 1-Lipschitz in ln m
    err = np.abs(np.log(m_gpu.cpu().numpy().astype(np.float64)) - np.log(m_ref))
    inside = (m_ref > lo) & (m_ref < hi)
    assert np.all(err <= 6.0 * sigma + 1e-5), (err.max(), sigma[np.argmax(err - 6 * sigma)])
    if scaled:
        # without the output scale the network sits below the mass floor and
        # every site is clamped; with it most sites are free
        assert inside.mean() > 0.5
        rms = np.sqrt(np.mean((err[inside] / sigma[inside]) ** 2))
        assert rms <= 1.5, rms
        assert np.max(err) > 1e-5


@pytest.mark.parametrize("batch,scaled", [(64, False), (4096, False), (4096, True)])
def test_gradient_matches_reference(rsv, ctx, problem, batch, scaled):
    params = dev(flat(problem["P"]), torch.float32)
    g, loss = rsv.rsv_mlp_grad(ctx, problem["F"], problem["target"], params, seed=11, step=3,
                               batch=batch, log_scale=problem["log_s_dev"] if scaled else None)
    idx = mlp.batch_indices(11, 3, problem["T"], batch)
    L, G = mlp.loss_and_grads(unflat(flat(problem["P"])), problem["Fnp"][idx],
                              problem["target_np"][idx], bf=True,
                              log_s=problem["log_s"] if scaled else 0.0)
    assert abs(loss.item() - L) <= 1e-4 * L
    gg = unflat(g.cpu().numpy())
    for k in G:
        scale = np.max(np.abs(G[k]))
        err = np.max(np.abs(gg[k] - G[k])) / scale
        assert err < 5e-3, (k, err)


def test_adam_steps_match_reference(rsv, ctx, problem):
    """Two GPU Adam steps against the reference Adam fed the GPU's own gradients."""
    params = dev(flat(problem["P"]), torch.float32)
    am = torch.zeros_like(params)
    av = torch.zeros_like(params)
    P = unflat(flat(problem["P"]))
    opt = mlp.Adam(P, lr=1e-3)
    for step in range(2):
        g, _ = rsv.rsv_mlp_grad(ctx, problem["F"], problem["target"], params, seed=1, step=step,
                                batch=512)
        rsv.rsv_mlp_train(ctx, problem["F"], problem["target"], params, am, av, step, 1, 512,
                          seed=1, lr=1e-3)
        opt.step(P, unflat(g.cpu().numpy()))
    got = params.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - flat(P).astype(np.float64))) < 2e-6


def test_training_reduces_loss_like_reference(rsv, ctx, problem):
    params = dev(flat(problem["P"]), torch.float32)
    am = torch.zeros_like(params)
    av = torch.zeros_like(params)
    losses = torch.empty(300, dtype=torch.float32, device="cuda")
    rsv.rsv_mlp_train(ctx, problem["F"], problem["target"], params, am, av, 0, 300, 1024,
                      seed=4, lr=3e-3, loss_out=losses)
    l = losses.cpu().numpy()
    assert l[-20:].mean() < 0.25 * l[:5].mean()
    P = unflat(flat(problem["P"]))
    opt = mlp.Adam(P, lr=3e-3)
    ref = []
    for step in range(300):
        idx = mlp.batch_indices(4, step, problem["T"], 1024)
        L, G = mlp.loss_and_grads(P, problem["Fnp"][idx], problem["target_np"][idx], bf=True)
        ref.append(L)
        opt.step(P, G)
    assert abs(l[-20:].mean() - np.mean(ref[-20:])) < 0.25 * np.mean(ref[-20:]) + 1e-3


def test_learned_mass_gains_over_identity(rsv, ctx):
    """The learned mass on a 2^16-site series, against the plain identity-mass
    sampler at its own settings (100 x 0.005): the posterior means of h agree
    within Monte-Carlo error, and the effective sample size per force
    evaluation (median over sites) is higher.  (On this posterior the learned
    m_t is close to the constant 1/Var(h_t); the gain is the larger stable
    step it allows.  ESS per second at 2^20 sites is reported by bench.py.)"""
    from paper_1603_08114_gb300 import learned
    T = 1 << 16
    s = synth.rsv_series(T, TH, seed=6)
    y, lr = dev(s.y), dev(s.lnrv)
    th = dev(TH)
    h = dev(s.h_true)
    mean, m2, cnt = learned.collect_moments(ctx, h, y, lr, th, 2000, 100, 0.005, seed=1)
    tm = learned.train_mass(ctx, y, lr, TH, mean, m2, cnt, steps=1000, batch=4096, lr=3e-3)
    losses = tm.losses.cpu().numpy()
    assert losses[-50:].mean() < 0.1 * losses[:10].mean()
    dt, n_md = learned.tune_step(ctx, h, y, lr, th, tm.minv, length=2.5)
    n = 400
    res = {}
    for name in ("identity", "mass"):
        hh = h.clone()
        snaps = torch.empty(n, T, dtype=torch.float32, device="cuda")
        if name == "identity":
            rsv.rsv_hmc_chain(ctx, hh, y, lr, th.clone(), 100, 0.005, n, prec="mixed", seed=3,
                              snaps=snaps, thin=1)
            grads = n * 100
        else:
            ms = learned.MassSampler(ctx, tm.minv, dt, n_md, 0.005, 100)
            ms.run(hh, y, lr, th.clone(), n, seed=3, snaps=snaps, update_theta=False)
            assert not ms.fell_back
            grads = n * n_md
        ess = rsv.rsv_ess(ctx, snaps).cpu().numpy()
        x = snaps.cpu().numpy().astype(np.float64)
        res[name] = dict(ess_per_grad=np.median(ess) / grads, mean=x.mean(0),
                         mcse=x.std(0) / np.sqrt(np.maximum(ess, 1)))
    z = np.abs(res["mass"]["mean"] - res["identity"]["mean"]) / np.sqrt(
        res["mass"]["mcse"] ** 2 + res["identity"]["mcse"] ** 2)
    assert np.mean(z < 3.5) > 0.99
    assert res["mass"]["ess_per_grad"] > res["identity"]["ess_per_grad"], (
        res["mass"]["ess_per_grad"], res["identity"]["ess_per_grad"], dt, n_md)


def test_trained_mass_recovers_exact_precision_in_gaussian_subcase(rsv, ctx):
    """y = 0: the posterior of h is Gaussian and 1/Var(h_t) is known exactly
    (tridiagonal inverse).  Trained on that exact target (output scale = its
    geometric mean) the network's m_t matches it within 3 % at every site,
    edges included."""
    from paper_1603_08114_gb300 import learned
    from tests.kalman_pin import tridiag_posterior
    T = 4000
    s = synth.rsv_series(T, TH, seed=8)
    y0 = np.zeros(T)
    m_exact, v_exact, _ = tridiag_posterior(s.lnrv, TH)
    target = dev(np.log(1.0 / v_exact).astype(np.float32), torch.float32)
    ls = dev([np.log(1.0 / v_exact).mean()], torch.float32)
    F, _ = rsv.rsv_mass_features(ctx, dev(y0), dev(s.lnrv), dev(m_exact), TH)
    params = dev(learned.glorot_params(0), torch.float32)
    am, av = torch.zeros_like(params), torch.zeros_like(params)
    rsv.rsv_mlp_train(ctx, F, target, params, am, av, 0, 3000, 1024, seed=5, lr=3e-3,
                      log_scale=ls)
    m = torch.empty(T, dtype=torch.float32, device="cuda")
    rsv.rsv_mlp_mass(ctx, F, params, dev(y0), dev(m_exact), TH, m_out=m, log_scale=ls)
    rel = np.abs(m.cpu().numpy() * v_exact - 1.0)
    assert np.max(rel) < 0.03, (np.max(rel), np.argmax(rel))


def test_fallback_to_identity_when_acceptance_collapses(rsv, ctx):
    from paper_1603_08114_gb300 import learned
    T = 4096
    s = synth.rsv_series(T, TH, seed=7)
    y, lr = dev(s.y), dev(s.lnrv)
    h = dev(s.h_true)
    bad = torch.full((T,), 400.0, dtype=torch.float32, device="cuda")  # step far too large
    ms = learned.MassSampler(ctx, bad, 0.3, 5, 0.005, 100, window=20)
    acc = torch.empty(60, dtype=torch.int32, device="cuda")
    ms.run(h, y, lr, dev(TH), 60, seed=2, accept_out=acc, update_theta=False)
    assert ms.fell_back
    assert acc[-20:].float().mean().item() > 0.6
