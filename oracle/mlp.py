"""FP64 oracle for the core-point surrogate network -- test infrastructure only.

The surrogate is a small multilayer perceptron d -> H -> H -> 1 with the exact
(erf) GELU, read as a logit for "this point is a core point".  The paper has no
learned component; this is the project's extension, and everything here is the
textbook definition written out in FP64 numpy:

  u  = (x - mean) / std                   input standardisation
  a1 = u W1^T + b1,   h1 = gelu(a1)       gelu(t) = t * Phi(t),  Phi = normal CDF
  a2 = h1 W2^T + b2,  h2 = gelu(a2)
  z  = h2 w3 + b3                         logit

  loss = mean_b [ max(z,0) - z*y + log(1 + exp(-|z|)) ]   (BCE with logits)

Backward is the chain rule of those lines (gelu'(t) = Phi(t) + t*phi(t)), and
the optimiser is Adam (Kingma & Ba 2015) with bias correction.

Pins (tests/test_oracle_mlp.py): central finite differences of ``loss`` for
every parameter tensor, GELU against Phi values from the error function,
BCE against its closed form at z = 0 (log 2), the first Adam step equal to
lr * sign(g) up to eps, three hand-worked Adam steps with changing gradients
(moments, both bias corrections and the updates, tests/golden/
adam_three_steps.txt), and training that drives the loss of a separable
problem down.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

PARAM_NAMES = ("w1", "b1", "w2", "b2", "w3", "b3")


def gelu(t):
    t = np.asarray(t, dtype=np.float64)
    return t * 0.5 * (1.0 + erf(t / math.sqrt(2.0)))


def gelu_grad(t):
    t = np.asarray(t, dtype=np.float64)
    cdf = 0.5 * (1.0 + erf(t / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * t * t) / math.sqrt(2.0 * math.pi)
    return cdf + t * pdf


def forward(params: dict, x, mean, std) -> dict:
    """Forward pass; returns every intermediate (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    u = (x - np.asarray(mean, np.float64)) / np.asarray(std, np.float64)
    w1, b1 = np.asarray(params["w1"], np.float64), np.asarray(params["b1"], np.float64)
    w2, b2 = np.asarray(params["w2"], np.float64), np.asarray(params["b2"], np.float64)
    w3, b3 = np.asarray(params["w3"], np.float64), float(np.asarray(params["b3"]).reshape(-1)[0])
    a1 = u @ w1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ w2.T + b2
    h2 = gelu(a2)
    z = h2 @ w3.reshape(-1) + b3
    return dict(u=u, a1=a1, h1=h1, a2=a2, h2=h2, z=z)


def bce_with_logits(z, y) -> float:
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss(params: dict, x, y, mean, std) -> float:
    return bce_with_logits(forward(params, x, mean, std)["z"], y)


def backward(params: dict, x, y, mean, std) -> tuple[float, dict]:
    """Loss and the gradient of the mean BCE loss w.r.t. every parameter."""
    f = forward(params, x, mean, std)
    y = np.asarray(y, dtype=np.float64)
    B = y.size
    z = f["z"]
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = (sig - y) / B                                   # d loss / d z
    w2 = np.asarray(params["w2"], np.float64)
    w3 = np.asarray(params["w3"], np.float64).reshape(-1)
    g = {}
    g["w3"] = f["h2"].T @ dz
    g["b3"] = np.array([dz.sum()])
    dh2 = np.outer(dz, w3)
    da2 = dh2 * gelu_grad(f["a2"])
    g["w2"] = da2.T @ f["h1"]
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ w2
    da1 = dh1 * gelu_grad(f["a1"])
    g["w1"] = da1.T @ f["u"]
    g["b1"] = da1.sum(axis=0)
    return bce_with_logits(z, y), g


def adam_step(params: dict, grads: dict, state: dict, lr=1e-3, beta1=0.9, beta2=0.999,
              eps=1e-8) -> dict:
    """One Adam update (Kingma & Ba 2015, Algorithm 1) in FP64 of every tensor
    named in ``grads``.  ``state`` holds ``t`` and the first/second moments;
    returns the new parameters."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = {}
    for k in grads:
        gk = np.asarray(grads[k], np.float64)
        mk = beta1 * state.get("m_" + k, np.zeros_like(gk)) + (1 - beta1) * gk
        vk = beta2 * state.get("v_" + k, np.zeros_like(gk)) + (1 - beta2) * gk * gk
        state["m_" + k], state["v_" + k] = mk, vk
        mhat = mk / (1 - beta1 ** t)
        vhat = vk / (1 - beta2 ** t)
        out[k] = np.asarray(params[k], np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return out
