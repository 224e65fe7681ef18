"""Pins for the FP64 surrogate-network oracle (oracle/mlp.py): finite
differences, closed forms of GELU / BCE / the first Adam step, three hand-worked Adam
steps, and the ARI."""
import math

import numpy as np
import pytest

from golden_io import read_kv
from oracle import mlp
from paper_2006_06743_gb300 import datagen


def _params(d=5, h=7, seed=0):
    p = datagen.mlp_init(d, h, seed)
    return {k: v.astype(np.float64) for k, v in p.items()}


def test_gelu_closed_forms():
    # gelu(t) = t * Phi(t); Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(-1.0) + 0.15865525393145707) < 1e-15
    assert mlp.gelu(0.0) == 0.0
    t = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.gelu(-t), mlp.gelu(t) - t, atol=1e-14)
    # derivative against central differences
    h = 1e-6
    fd = (mlp.gelu(t + h) - mlp.gelu(t - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(t), fd, atol=1e-8)


def test_bce_closed_forms():
    assert abs(mlp.bce_with_logits([0.0], [1.0]) - math.log(2.0)) < 1e-15
    assert abs(mlp.bce_with_logits([0.0], [0.0]) - math.log(2.0)) < 1e-15
    z = 3.0
    assert abs(mlp.bce_with_logits([z], [1.0]) - math.log1p(math.exp(-z))) < 1e-15
    assert abs(mlp.bce_with_logits([z], [0.0]) - (z + math.log1p(math.exp(-z)))) < 1e-14
    # no overflow at large |z|
    assert abs(mlp.bce_with_logits([800.0], [0.0]) - 800.0) < 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_finite_differences(seed):
    d, h, B = 5, 7, 9
    p = _params(d, h, seed)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, d))
    y = (rng.uniform(size=B) < 0.5).astype(np.float64)
    mean, std = x.mean(0), x.std(0) + 0.5
    L, g = mlp.backward(p, x, y, mean, std)
    assert abs(L - mlp.loss(p, x, y, mean, std)) < 1e-14
    eps = 1e-6
    for k in mlp.PARAM_NAMES:
        flat = p[k].reshape(-1)
        fd = np.empty_like(flat)
        for t in range(flat.size):
            old = flat[t]
            flat[t] = old + eps
            lp = mlp.loss(p, x, y, mean, std)
            flat[t] = old - eps
            lm = mlp.loss(p, x, y, mean, std)
            flat[t] = old
            fd[t] = (lp - lm) / (2 * eps)
        np.testing.assert_allclose(np.asarray(g[k]).reshape(-1), fd, rtol=1e-6, atol=1e-9,
                                   err_msg=k)


def test_adam_first_step_is_lr_sign():
    p = _params()
    g = {k: np.full_like(v, 0.3) * np.sign(np.arange(v.size).reshape(v.shape) % 2 - 0.5)
         for k, v in p.items()}
    st = {}
    q = mlp.adam_step(p, g, st, lr=1e-3)
    for k in mlp.PARAM_NAMES:
        step = p[k] - q[k]
        np.testing.assert_allclose(step, 1e-3 * np.sign(g[k]) * (0.3 / (0.3 + 1e-8)),
                                   rtol=1e-9)
    assert st["t"] == 1


def test_adam_three_hand_worked_steps():
    """Three Adam steps with a different gradient each time, against the
    hand-worked moments, bias corrections and updates of
    tests/golden/adam_three_steps.txt (exact fractions)."""
    from fractions import Fraction as Fr
    kv = read_kv("adam_three_steps.txt")
    lr, b1, b2 = (float(Fr(kv[k][0])) for k in ("lr", "beta1", "beta2"))
    theta = np.array([float(Fr(v)) for v in kv["theta0"]])
    st = {}
    for t in (1, 2, 3):
        row = [Fr(v) for v in kv[f"step{t}"]]
        g, m, v, mhat, vhat = (np.array([float(a), float(b)]) for a, b in
                               zip(row[0::2], row[1::2]))
        q = mlp.adam_step({"w": theta}, {"w": g}, st, lr=lr, beta1=b1, beta2=b2, eps=0.0)
        assert st["t"] == t
        np.testing.assert_allclose(st["m_w"], m, rtol=1e-15, atol=0)
        np.testing.assert_allclose(st["v_w"], v, rtol=1e-15, atol=0)
        np.testing.assert_allclose(st["m_w"] / (1 - b1 ** t), mhat, rtol=1e-14)
        np.testing.assert_allclose(st["v_w"] / (1 - b2 ** t), vhat, rtol=1e-14)
        np.testing.assert_allclose(theta - q["w"], lr * mhat / np.sqrt(vhat), rtol=1e-13)
        theta = q["w"]


def test_training_reduces_loss():
    d, h = 4, 16
    p = _params(d, h, 3)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((256, d))
    y = (x[:, 0] + 0.5 * x[:, 1] > 0).astype(np.float64)
    mean, std = x.mean(0), x.std(0)
    st = {}
    l0 = mlp.loss(p, x, y, mean, std)
    for _ in range(200):
        _, g = mlp.backward(p, x, y, mean, std)
        p = mlp.adam_step(p, g, st, lr=1e-2)
    assert mlp.loss(p, x, y, mean, std) < 0.3 * l0


def test_ari_hand_case(orc):
    kv = read_kv("ari_hand.txt")
    a = [int(v) for v in kv["a"]]
    b = [int(v) for v in kv["b"]]
    want = int(kv["ari_num"][0]) / int(kv["ari_den"][0])
    assert abs(orc.ari(a, b) - want) < 1e-15
    assert orc.ari(a, a) == 1.0
    # invariant under relabelling
    assert abs(orc.ari([5, 5, 5, -1, -1, -1], b) - want) < 1e-15


def test_ari_matches_sklearn(orc):
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(8)
    for _ in range(5):
        a = rng.integers(-1, 6, size=500)
        b = np.where(rng.uniform(size=500) < 0.7, a, rng.integers(-1, 9, size=500))
        assert abs(orc.ari(a, b) - skm.adjusted_rand_score(a, b)) < 1e-12


def test_canonical_relabel(orc):
    lab = np.array([7, 7, -1, 3, 7, 3])
    np.testing.assert_array_equal(orc.canonical(lab), [0, 0, -1, 3, 0, 3])
