"""The learned surrogate: its kernels against the FP64 network oracle
(forward, loss, every gradient), training that reduces the loss, the gated
clustering against the oracle's gated form of Algorithm 1, and what the
trained network gains over the plain method on a sibling dataset."""
import numpy as np
import pytest

from gpu_util import need_gpu
from oracle import mlp as omlp
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _fp16(p: dict) -> dict:
    return {k: np.asarray(v, np.float32).astype(np.float16).astype(np.float64)
            for k, v in p.items()}


def _setup(d, n, seed):
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import surrogate as sg
    init = datagen.mlp_init(d, 128, seed)
    net = sg.Surrogate(init)
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((n, d)) * 2 + 1).astype(np.float32)
    y = (rng.uniform(size=n) < 0.4).astype(np.uint8)
    xg = torch.from_numpy(x).cuda()
    yg = torch.from_numpy(y).cuda()
    net.standardize(xg)
    _, mean, std = sg.unpack(net.params.cpu().numpy(), d)
    return torch, sng, sg, net, init, x, y, xg, yg, mean, std


@pytest.mark.parametrize("d,n", [(5, 37), (32, 200), (64, 130), (2, 64), (17, 1000),
                                 (48, 3001)])
def test_standardize_and_forward_match_oracle(d, n):
    """Inference against the FP64 network on the same FP16-rounded weights.
    CUDA-core path (FP32 activations): |dp| <= 2e-5.  Tensor-core path: the
    standardised inputs and the layer-1 outputs are rounded to FP16 at the MMA
    inputs (relative 2^-11 each), which moves the logit by ~5e-4 on sums of
    <= 128 terms of weights ~0.1 (|dp| <= |dz| / 4); bound used: 2e-3, for
    the warp-level MMA path and the tcgen05 path alike."""
    torch, sng, sg, net, init, x, y, xg, yg, mean, std = _setup(d, n, d)
    np.testing.assert_allclose(mean, x.astype(np.float64).mean(0), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(std, x.astype(np.float64).std(0), rtol=1e-5, atol=1e-5)
    f = omlp.forward(_fp16(init), x, mean.astype(np.float64), std.astype(np.float64))
    want = 1.0 / (1.0 + np.exp(-f["z"]))
    net.cfg.fp32_activations = 1
    np.testing.assert_allclose(net.predict(xg).cpu().numpy(), want, atol=2e-5)
    net.cfg.fp32_activations = 0
    np.testing.assert_allclose(net.predict(xg).cpu().numpy(), want, atol=2e-3)
    # the tcgen05 path: the same FP16 operands, accumulators in tensor memory
    net.cfg.fp32_activations = 2
    np.testing.assert_allclose(net.predict(xg).cpu().numpy(), want, atol=2e-3)


@pytest.mark.parametrize("d,n", [(5, 37), (32, 256), (64, 100)])
def test_loss_and_gradients_match_oracle(d, n):
    """Analytic FP64 backprop of the oracle (itself pinned by finite
    differences) against the FP32 kernels, on the same FP16-rounded weights.
    Tolerance: FP32 sums of at most ~300 terms per layer, three layers deep."""
    torch, sng, sg, net, init, x, y, xg, yg, mean, std = _setup(d, n, 100 + d)
    loss, g = net.loss_grad(xg, yg)
    L, G = omlp.backward(_fp16(init), x, y.astype(np.float64), mean.astype(np.float64),
                         std.astype(np.float64))
    assert abs(loss - L) < 1e-5 * max(1.0, abs(L))
    got, _, _ = sg.unpack(np.concatenate([g.cpu().numpy(), np.zeros(2 * d, np.float32)]), d)
    for k in omlp.PARAM_NAMES:
        want = np.asarray(G[k]).reshape(got[k].shape)
        scale = np.abs(want).max() + 1e-12
        np.testing.assert_allclose(got[k], want, rtol=2e-3, atol=2e-4 * scale, err_msg=k)


def test_training_reduces_loss_and_learns_a_rule():
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import surrogate as sg
    d, n = 8, 50_000
    rng = np.random.default_rng(3)
    x = rng.standard_normal((n, d)).astype(np.float32)
    y = ((x[:, 0] ** 2 + x[:, 1] ** 2) < 1.0).astype(np.uint8)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net = sg.Surrogate(datagen.mlp_init(d, 128, 1), cfg=sg.TrainConfig(batch=512, lr=3e-3))
    net.standardize(xg)
    trace = net.train(xg, yg, 600)
    assert trace[-50:].mean() < 0.5 * trace[:10].mean()
    acc = ((net.predict(xg).cpu().numpy() > 0.5) == y.astype(bool)).mean()
    assert acc > 0.95


def test_training_steps_match_oracle_adam():
    """Three full-batch steps through sng_mlp_train (rows taken in order)
    equal the oracle's Adam (Kingma & Ba 2015) applied to the gradients that
    sng_mlp_loss_grad reports at each step's parameters."""
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import surrogate as sg
    d, n = 6, 300
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, d)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    init = datagen.mlp_init(d, 128, 9)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net = sg.Surrogate(init, cfg=sg.TrainConfig(batch=n, lr=1e-3, sequential=True))
    net.standardize(xg)
    nt = sg.trained_count(d)
    state = {}
    for _ in range(3):
        p0 = net.params.clone()
        _, g = net.loss_grad(xg, yg)
        net.train(xg, yg, 1)
        q = omlp.adam_step({"w": p0[:nt].double().cpu().numpy()},
                           {"w": g.double().cpu().numpy()}, state, lr=1e-3)
        np.testing.assert_allclose(net.params[:nt].cpu().numpy(), q["w"], rtol=1e-5, atol=1e-7)
        assert torch.equal(net.params[nt:], p0[nt:])


def _clear_threshold(prob, target: float, tol: float, span: float) -> float:
    """A float32 threshold within ``span`` of ``target`` with as few oracle
    probabilities as possible within ``tol`` of it (the kernels'
    probabilities are within ``tol`` of the oracle's), nearest to ``target``
    among those; 0 and 1 stay (nothing lies below 0 or above 1)."""
    if target <= 0.0 or target >= 1.0:
        return target
    lo, hi = max(target - span, 1e-6), min(target + span, 1.0 - 1e-6)
    srt = np.sort(prob)
    inside = srt[(srt > lo) & (srt < hi)]
    cand = np.concatenate([np.linspace(lo, hi, 4001), 0.5 * (inside[1:] + inside[:-1])])
    cand = np.float32(cand)
    cand = cand[(cand > 0) & (cand < 1)].astype(np.float64)
    near = (np.searchsorted(srt, cand + tol, side="right")
            - np.searchsorted(srt, cand - tol, side="left"))
    best = near.min()
    pick = cand[near == best]
    return float(pick[np.argmin(np.abs(pick - target))])


def _gate_variants(prob, tol, m, pn, pc, frac, nfrac, rw, orc, limit=4, by_degree=False):
    """The oracle's gate decisions, and, for the few points whose oracle
    probability lies within ``tol`` of a threshold (where the kernels may fall
    either way), every combination of their two possible decisions."""
    near = np.zeros(prob.size, bool)
    for t in (pn, pc):
        if 0.0 < t < 1.0:               # nothing is below 0 or above 1
            near |= np.abs(prob - t) <= tol
    amb = np.flatnonzero(near)
    assert amb.size <= limit, f"{amb.size} points within {tol} of a threshold"
    out = []
    for bits in range(1 << amb.size):
        q = prob.copy()
        for k, idx in enumerate(amb):
            t = pn if abs(prob[idx] - pn) <= tol else pc
            q[idx] = t + 4 * tol if (bits >> k) & 1 else t - 4 * tol
        out.append(orc.gate_decisions(q, m, pn, pc, frac, nfrac, rw, by_degree=by_degree))
    return out


@pytest.mark.parametrize("n,fp32_act,form", [(2000, 0, "plain"), (2000, 2, "plain"),
                                             (6000, 1, "plain"), (400_000, 1, "plain"),
                                             (6000, 1, "mma"), (6000, 1, "tc05"),
                                             (6000, 1, "fp8")])
def test_gated_cluster_matches_oracle_gated_form(orc, n, fp32_act, form):
    """The surrogate path against the oracle's gated form of Algorithm 1, with
    every expected value from the oracle: the gate's probabilities from the
    FP64 network oracle on the trained network's FP16-rounded weights, its
    decisions from the oracle's gate rule, the clustering from the oracle's
    gated form.  Thresholds are moved to a nearby place with as few oracle
    probabilities as possible within the kernels' stated error of them (2e-5
    with FP32 activations, 2e-3 on tensor cores); the at most four points
    left there may be decided either way, and the result must equal the
    oracle's for one of those combinations.  At n = 400,000 the gather runs one lane per row, with
    per-row draw counts and weights; the screened forms (tensor-core BF16,
    TMA + tcgen05, FP8 copy) take the same per-row counts and weights."""
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import surrogate as sg
    d, m = 8, 120
    x = datagen.gaussian_mixture(n, d, 8, 0.05, seed=2, centre_std=1.0, sigma_lo=0.05,
                                 sigma_hi=0.1)
    eps = datagen.eps_quantile(x, 0.05, 200_000, seed=2)
    xg = torch.from_numpy(x).cuda()
    flags = {"plain": 0, "mma": sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA,
             "tc05": sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA | sng.SNG_FLAG_TCGEN05,
             "fp8": sng.SNG_FLAG_SCREEN8}[form]
    want_screen = {"plain": 0, "mma": 2, "tc05": 3, "fp8": 4}[form]
    p = sng.Params(eps=eps, min_pts=5, m=m, seed=4, flags=flags)
    plain, plain_core, _ = sng.cluster(xg, p, want_core=True)
    net = sg.Surrogate(datagen.mlp_init(d, 128, 2), cfg=sg.TrainConfig(batch=1024, lr=3e-3))
    net.standardize(xg)
    net.train(xg, plain_core, 300)
    net.cfg.fp32_activations = fp32_act
    tol = 2e-5 if fp32_act == 1 else 2e-3
    w, mean, std = sg.unpack(net.params.cpu().numpy(), d)
    f = omlp.forward(_fp16(w), x, mean.astype(np.float64), std.astype(np.float64))
    prob = 1.0 / (1.0 + np.exp(-f["z"]))
    for pn, pc, frac, nfrac, rw, bd in ((0.1, 0.9, 0.25, 0.0, False, False),
                                        (0.3, 0.6, 0.5, 0.0, False, False),
                                        (0.0, 1.0, 0.25, 0.0, False, False),
                                        (0.1, 0.9, 0.25, 0.1, True, False),
                                        (0.05, 0.95, 0.3, 0.5, True, False),
                                        (0.2, 0.8, 0.5, 0.0, True, False),
                                        (0.1, 0.9, 0.25, 0.25, True, True),
                                        (0.2, 0.7, 0.5, 0.0, True, True)):
        span = min(0.2, 0.45 * (pc - pn))       # keeps p_noise below p_core
        pn, pc = _clear_threshold(prob, pn, tol, span), _clear_threshold(prob, pc, tol, span)
        assert pn <= pc
        labels, core, st = net.cluster(xg, p, pn, pc, frac, nfrac, rw, want_core=True,
                                       by_degree=bd)
        assert st["map_screen"] == want_screen
        got_l, got_c = labels.cpu().numpy(), core.cpu().numpy()
        match = False
        for forced, m_row, w_row in _gate_variants(prob, tol, m, pn, pc, frac, nfrac, rw, orc,
                                                   by_degree=bd):
            r = orc.cluster_gated(x, eps, p.seed, m, p.min_pts, forced, m_row, w_row=w_row)
            if (np.array_equal(got_c, r["core"]) and np.array_equal(got_l, r["labels"])
                    and st["queries"] == r["queries"]
                    and (bd or (st["surrogate_core"] == int((forced == 1).sum())
                                and st["surrogate_noise"] == int((forced == 2).sum())))):
                match = True
                break
        assert match, (pn, pc, frac, nfrac, rw)
    # nothing gated: the plain method exactly
    labels, _ = net.cluster(xg, p, 0.0, 1.0, 0.25)
    assert torch.equal(labels, plain)


def test_surrogate_gain_on_sibling_dataset():
    """The learned-surrogate configuration (n = 2,000,000 points in d = 32
    from a 200-Gaussian mixture with 3% noise, m = 1000, eps = 1% distance
    quantile, MinPts = 8), trained on core masks of ten sibling datasets: on a
    fresh sibling, with points of confidence above 0.9 declared core and
    drawing three quarters of their partners, the gate removes over a tenth of
    the sampled queries while its clustering stays within ARI >= 0.99 and
    core-mask agreement >= 0.99 of the plain method's on the same draws.
    (For scale: the plain method against itself with another seed gives ARI
    ~0.78 on this data.)"""
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import surrogate as sg
    n, d, m = 2_000_000, 32, 1000
    master = 4242
    xs, ys = [], []
    eps = None
    for k in range(11):
        x = datagen.gaussian_mixture(n, d, 200, 0.03, seed=100 + k, master_seed=master)
        if eps is None:
            eps = datagen.eps_quantile(x, 0.01, 1_000_000, seed=0)
        xg = torch.from_numpy(x).cuda()
        _, core, _ = sng.cluster(xg, sng.Params(eps=eps, min_pts=8, m=m, seed=k), want_core=True)
        xs.append(xg)
        ys.append(core)
    x_test = xs.pop()
    ys.pop()
    xtr = torch.cat(xs).contiguous()
    ytr = torch.cat(ys).contiguous()
    del xs, ys
    net = sg.Surrogate(datagen.mlp_init(d, 128, 5), cfg=sg.TrainConfig(batch=4096, lr=1e-3))
    net.standardize(xtr)
    trace = net.train(xtr, ytr, 3000)
    assert trace[-200:].mean() < 0.5 * trace[:20].mean()
    p = sng.Params(eps=eps, min_pts=8, m=m, seed=77)
    plain, plain_core, pst = sng.cluster(x_test, p, want_core=True)
    labels, core, st = net.cluster(x_test, p, p_noise=0.0, p_core=0.9, core_draw_frac=0.75,
                                   want_core=True)
    ari = sng.ari(labels, plain)
    agree = (core == plain_core).float().mean().item()
    assert st["queries"] < 0.9 * pst["queries"], (st["queries"], pst["queries"])
    assert ari >= 0.99, ari
    assert agree >= 0.99, agree


def test_checkpoint_resume_is_exact(tmp_path):
    """A network saved mid-training and loaded back predicts identically, and
    training resumed from the checkpoint (Adam state and step included)
    matches training continued in place."""
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import surrogate as sg
    d, n = 8, 20_000
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, d)).astype(np.float32)
    y = (x[:, 0] + 0.5 * x[:, 1] > 0).astype(np.uint8)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    cfg = sg.TrainConfig(batch=512, lr=3e-3)
    net = sg.Surrogate(datagen.mlp_init(d, 128, 1), cfg=cfg)
    net.standardize(xg)
    net.train(xg, yg, 50)
    path = str(tmp_path / "net.bin")
    net.save(path)
    back = sg.Surrogate.load(path, cfg=cfg)
    assert back.step == net.step
    assert torch.equal(back.predict(xg), net.predict(xg))
    la = net.train(xg, yg, 20)
    lb = back.train(xg, yg, 20)
    np.testing.assert_array_equal(la, lb)
    assert torch.equal(back.params, net.params)
