"""Core-point surrogate: training and gated clustering through libsng.so.

A d -> 128 -> 128 -> 1 perceptron (exact GELU, FP16-rounded weights, FP32
accumulation) learns, from coordinates alone, the core mask that Algorithm 1
(Jiang, Jang & Lacki 2020, Section 3, step 3) produces on sibling datasets
drawn from the same distribution.  At clustering time the network gates each
point: confidently non-core points draw no partners, confidently core points
draw a prefix of their partner stream, and the rest run the full sampled
queries.  Every arithmetic step runs in the library's CUDA kernels; this
module packs parameters and drives the calls.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import (SNG_F32, Params, _check, _rows, _stream_ptr, lib, sng_gate, sng_mlp_config,
               sng_stats)

HIDDEN = 128


def param_count(d: int) -> int:
    return int(lib().sng_mlp_param_count(d, HIDDEN))


def trained_count(d: int) -> int:
    return param_count(d) - 2 * d


def pack(p: dict, mean=None, std=None) -> np.ndarray:
    """Flat FP32 parameter vector in the library's layout."""
    d = p["w1"].shape[1]
    mean = np.zeros(d, np.float32) if mean is None else np.asarray(mean, np.float32)
    std = np.ones(d, np.float32) if std is None else np.asarray(std, np.float32)
    v = np.concatenate([np.asarray(p[k], np.float32).ravel()
                        for k in ("w1", "b1", "w2", "b2", "w3", "b3")] + [mean, std])
    assert v.size == param_count(d)
    return v


def unpack(v, d: int) -> tuple[dict, np.ndarray, np.ndarray]:
    v = np.asarray(v, np.float32)
    H = HIDDEN
    o = 0
    out = {}
    for k, shape in (("w1", (H, d)), ("b1", (H,)), ("w2", (H, H)), ("b2", (H,)),
                     ("w3", (H,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[k] = v[o:o + size].reshape(shape)
        o += size
    return out, v[o:o + d], v[o + d:o + 2 * d]


# ------------------------------------------------------------ checkpoints
#
# File layout (little-endian): the 8-byte magic b"SNGMLP01", then int32
# version (1), d, hidden, parameter count P, trained count T, flags (bit 0:
# Adam moments follow), int64 Adam step, then P FP32 parameters in the
# library's layout (w1, b1, w2, b2, w3, b3, mean, std) and, with bit 0, the T
# FP32 first moments and T FP32 second moments.

MAGIC = b"SNGMLP01"
_HEADER = np.dtype([("version", "<i4"), ("d", "<i4"), ("hidden", "<i4"), ("n_params", "<i4"),
                    ("n_trained", "<i4"), ("flags", "<i4"), ("step", "<i8")])


def _counts(d: int, hidden: int = HIDDEN) -> tuple[int, int]:
    trained = hidden * d + hidden + hidden * hidden + hidden + hidden + 1
    return trained + 2 * d, trained


def save_params(path: str, params, d: int, step: int = 0, m=None, v=None) -> None:
    """Write a parameter vector (and optionally Adam moments) to ``path``."""
    n_params, n_trained = _counts(d)
    params = np.ascontiguousarray(params, dtype="<f4").ravel()
    if params.size != n_params:
        raise ValueError(f"expected {n_params} parameters for d = {d}, got {params.size}")
    moments = m is not None and v is not None
    hdr = np.zeros(1, dtype=_HEADER)
    hdr[0] = (1, d, HIDDEN, n_params, n_trained, 1 if moments else 0, step)
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(hdr.tobytes())
        f.write(params.tobytes())
        if moments:
            for a in (m, v):
                a = np.ascontiguousarray(a, dtype="<f4").ravel()
                if a.size != n_trained:
                    raise ValueError(f"expected {n_trained} moments, got {a.size}")
                f.write(a.tobytes())


def load_params(path: str) -> dict:
    """Read a file written by ``save_params``: d, step, params, and m / v
    (None when the file holds no moments).  Raises ValueError on a wrong
    magic, version, size or truncated file."""
    with open(path, "rb") as f:
        blob = f.read()
    if blob[:8] != MAGIC:
        raise ValueError("not a surrogate checkpoint (bad magic)")
    if len(blob) < 8 + _HEADER.itemsize:
        raise ValueError("truncated checkpoint header")
    hdr = np.frombuffer(blob, dtype=_HEADER, count=1, offset=8)[0]
    if int(hdr["version"]) != 1 or int(hdr["hidden"]) != HIDDEN:
        raise ValueError("unsupported checkpoint version or hidden width")
    d = int(hdr["d"])
    n_params, n_trained = _counts(d)
    if int(hdr["n_params"]) != n_params or int(hdr["n_trained"]) != n_trained:
        raise ValueError("checkpoint sizes do not match its d")
    moments = bool(int(hdr["flags"]) & 1)
    need = 8 + _HEADER.itemsize + 4 * (n_params + (2 * n_trained if moments else 0))
    if len(blob) != need:
        raise ValueError(f"checkpoint is {len(blob)} bytes, expected {need}")
    o = 8 + _HEADER.itemsize
    params = np.frombuffer(blob, dtype="<f4", count=n_params, offset=o).astype(np.float32)
    m = v = None
    if moments:
        o += 4 * n_params
        m = np.frombuffer(blob, dtype="<f4", count=n_trained, offset=o).astype(np.float32)
        v = np.frombuffer(blob, dtype="<f4", count=n_trained,
                          offset=o + 4 * n_trained).astype(np.float32)
    return {"d": d, "step": int(hdr["step"]), "params": params, "m": m, "v": v}


@dataclass
class TrainConfig:
    batch: int = 4096
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    seed: int = 0
    sequential: bool = False
    fp32_activations: int = 0   # 0 mma.sync, 1 FP32 CUDA cores, 2 tcgen05

    def to_c(self, d: int) -> sng_mlp_config:
        c = sng_mlp_config()
        c.d, c.hidden, c.batch = d, HIDDEN, self.batch
        c.lr, c.beta1, c.beta2, c.adam_eps = self.lr, self.beta1, self.beta2, self.adam_eps
        c.seed = self.seed & (2**64 - 1)
        c.sequential = int(self.sequential)
        c.fp32_activations = int(self.fp32_activations)
        return c


class Surrogate:
    """Device-resident network state (parameters and Adam moments)."""

    def __init__(self, init: dict, device="cuda", cfg: TrainConfig | None = None):
        import torch
        self.d = init["w1"].shape[1]
        self.cfg = cfg or TrainConfig()
        self.params = torch.from_numpy(pack(init)).to(device)
        nt = trained_count(self.d)
        self.m = torch.zeros(nt, dtype=torch.float32, device=device)
        self.v = torch.zeros(nt, dtype=torch.float32, device=device)
        self.step = 0

    def save(self, path: str, optimizer: bool = True) -> None:
        """Checkpoint the parameters (and the Adam state) to ``path``."""
        m, v = (self.m.cpu().numpy(), self.v.cpu().numpy()) if optimizer else (None, None)
        save_params(path, self.params.cpu().numpy(), self.d, self.step, m, v)

    @classmethod
    def load(cls, path: str, device="cuda", cfg: TrainConfig | None = None) -> "Surrogate":
        """A network restored from ``save``; training resumes from its Adam
        state and step when the file holds them."""
        import torch
        ck = load_params(path)
        net = cls.__new__(cls)
        net.d = ck["d"]
        net.cfg = cfg or TrainConfig()
        net.params = torch.from_numpy(ck["params"]).to(device)
        nt = _counts(net.d)[1]
        net.m = (torch.from_numpy(ck["m"]).to(device) if ck["m"] is not None
                 else torch.zeros(nt, dtype=torch.float32, device=device))
        net.v = (torch.from_numpy(ck["v"]).to(device) if ck["v"] is not None
                 else torch.zeros(nt, dtype=torch.float32, device=device))
        net.step = ck["step"]
        return net

    def standardize(self, x):
        _rows(x, SNG_F32)
        _check(lib().sng_mlp_standardize(x.data_ptr(), x.shape[0], self.d,
                                         self.params.data_ptr(), _stream_ptr()))

    def train(self, x, y, steps: int):
        """``steps`` Adam steps on hash-sampled batches of (x, y); returns the
        per-step batch losses (float32 numpy)."""
        import torch
        assert x.is_contiguous() and y.dtype == torch.uint8
        trace = torch.empty(max(1, steps), dtype=torch.float32, device=x.device)
        c = self.cfg.to_c(self.d)
        _check(lib().sng_mlp_train(x.data_ptr(), y.data_ptr(), x.shape[0], ctypes.byref(c),
                                   self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                   self.step, steps, trace.data_ptr(), _stream_ptr()))
        self.step += steps
        return trace[:steps].cpu().numpy()

    def loss_grad(self, x, y):
        import torch
        g = torch.empty(trained_count(self.d), dtype=torch.float32, device=x.device)
        loss = ctypes.c_double()
        c = self.cfg.to_c(self.d)
        _check(lib().sng_mlp_loss_grad(x.data_ptr(), y.data_ptr(), x.shape[0], ctypes.byref(c),
                                       self.params.data_ptr(), g.data_ptr(), ctypes.byref(loss),
                                       _stream_ptr()))
        return float(loss.value), g

    def predict(self, x):
        import torch
        prob = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        c = self.cfg.to_c(self.d)
        _check(lib().sng_mlp_predict(x.data_ptr(), x.shape[0], ctypes.byref(c),
                                     self.params.data_ptr(), prob.data_ptr(), _stream_ptr()))
        return prob

    def cluster(self, x, p: Params, p_noise: float = 0.0, p_core: float = 0.95,
                core_draw_frac: float = 0.5, noise_draw_frac: float = 0.0,
                reweight: bool = False, want_core: bool = False, by_degree: bool = False):
        """Algorithm 1 gated by this network; returns (labels[, core], stats).
        ``by_degree``: the gate only sets draw budgets; every point keeps the
        degree test (use with ``reweight``)."""
        import torch
        n, d, ld = _rows(x, SNG_F32)
        labels = torch.empty(n, dtype=torch.int32, device=x.device)
        core = torch.empty(n, dtype=torch.uint8, device=x.device) if want_core else None
        st = sng_stats()
        c = self.cfg.to_c(self.d)
        g = sng_gate()
        g.p_noise, g.p_core = p_noise, p_core
        g.core_draw_frac, g.noise_draw_frac, g.reweight = core_draw_frac, noise_draw_frac, int(reweight)
        g.by_degree = int(by_degree)
        _check(lib().sng_cluster_surrogate(
            x.data_ptr(), ctypes.byref(p.to_c(n, d, ld, SNG_F32)), ctypes.byref(c),
            self.params.data_ptr(), ctypes.byref(g), labels.data_ptr(),
            core.data_ptr() if core is not None else None, ctypes.byref(st), _stream_ptr()))
        out = st.as_dict()
        return (labels, core, out) if want_core else (labels, out)
