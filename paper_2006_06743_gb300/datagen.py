"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no partner hash, no eps-test, no graph step), so both the
CUDA path and the FP64 oracle can take their inputs from it.  Every generator
uses numpy's PCG64 stream seeded by the caller, returns C-contiguous float32
rows, and states its recipe in its docstring.

The paper evaluates on UCI/OpenML datasets of n ~ 1e6 points in D = 3..411
(Section 5, Figures 2 and 8); those are not available here, and these mixtures
stand in for them with the sizes, dimensions, sampling rates and MinPts the
benchmark configurations fix.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def mixture_2d(n: int = 10_000, k: int = 5, sigma: float = 0.05, noise_frac: float = 0.05,
               seed: int = 0) -> np.ndarray:
    """(1 - noise_frac) of the points from k isotropic 2-D Gaussians with equal
    weights (std sigma, centres uniform in [0,1]^2); the rest uniform on
    [0,1]^2.  Rows are shuffled."""
    rng = _rng(seed)
    n_noise = int(round(noise_frac * n))
    n_cl = n - n_noise
    centres = rng.uniform(0.0, 1.0, size=(k, 2))
    which = rng.integers(0, k, size=n_cl)
    pts = centres[which] + sigma * rng.standard_normal((n_cl, 2))
    noise = rng.uniform(0.0, 1.0, size=(n_noise, 2))
    x = np.concatenate([pts, noise]).astype(np.float32)
    return np.ascontiguousarray(x[rng.permutation(n)])


def gaussian_mixture(n: int, d: int, k: int, noise_frac: float, seed: int,
                     centre_std: float = 2.0, sigma_lo: float = 0.5, sigma_hi: float = 1.0,
                     master_seed: int | None = None, return_truth: bool = False):
    """High-dimensional mixture: k Gaussian clusters with centres N(0, centre_std^2 I),
    per-cluster std uniform in [sigma_lo, sigma_hi], cluster sizes from
    Dirichlet(alpha = 1) weights, plus noise_frac of the points uniform in the
    bounding box of the clustered points.  Rows are shuffled.

    ``master_seed`` (default: ``seed``) fixes the mixture itself (centres,
    stds, weights); ``seed`` draws the sample, so sibling datasets share one
    distribution.  ``return_truth`` also returns the generating component of
    each row (-1 for noise)."""
    master = _rng(seed if master_seed is None else master_seed)
    centres = centre_std * master.standard_normal((k, d))
    sig = master.uniform(sigma_lo, sigma_hi, size=k)
    w = master.dirichlet(np.ones(k))
    rng = _rng(seed + 0x5EED if master_seed is not None else seed ^ 0x5EED)
    n_noise = int(round(noise_frac * n))
    n_cl = n - n_noise
    counts = rng.multinomial(n_cl, w)
    which = np.repeat(np.arange(k), counts)
    x = np.empty((n, d), dtype=np.float32)
    z = rng.standard_normal((n_cl, d), dtype=np.float32)
    x[:n_cl] = (centres[which] + sig[which, None] * z).astype(np.float32)
    lo = x[:n_cl].min(axis=0)
    hi = x[:n_cl].max(axis=0)
    x[n_cl:] = rng.uniform(lo, hi, size=(n_noise, d)).astype(np.float32)
    truth = np.concatenate([which, -np.ones(n_noise, dtype=np.int64)])
    perm = rng.permutation(n)
    x = np.ascontiguousarray(x[perm])
    if return_truth:
        return x, truth[perm]
    return x


def sphere_embeddings(n: int, d: int, n_centres: int, sigma: float, seed: int) -> np.ndarray:
    """Unit-norm embedding-like vectors: n_centres centres uniform on the unit
    sphere S^{d-1}; each point is a random centre plus N(0, sigma^2 I), then
    renormalised to unit length.  Generated in chunks to bound host memory."""
    rng = _rng(seed)
    c = rng.standard_normal((n_centres, d))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    c = c.astype(np.float32)
    x = np.empty((n, d), dtype=np.float32)
    chunk = 1 << 20
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        which = rng.integers(0, n_centres, size=e - s)
        v = c[which] + np.float32(sigma) * rng.standard_normal((e - s, d), dtype=np.float32)
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x[s:e] = v
    return x


def uniform_balls(n: int, seed: int, centres=((0.0, 0.0, 0.0), (3.0, 0.0, 0.0),
                                              (0.0, 3.0, 0.0)), radius: float = 1.0):
    """Uniform mixture of balls in R^3 (the simulation of the paper's Figure 1):
    each point picks a ball uniformly and is uniform inside it.  Returns the
    points and the generating ball of each point."""
    rng = _rng(seed)
    c = np.asarray(centres, dtype=np.float64)
    which = rng.integers(0, len(c), size=n)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    x = (c[which] + v * r[:, None]).astype(np.float32)
    return np.ascontiguousarray(x), which


def point_clouds(n_clouds: int, seed: int, n_min: int = 2000, n_max: int = 130_000,
                 blobs_min: int = 5, blobs_max: int = 60, sigma_lo: float = 0.1,
                 sigma_hi: float = 0.5, box=(100.0, 100.0, 4.0), ground_frac: float = 0.3,
                 ground_sigma: float = 0.05, pad_to: int = 4):
    """Batch of independent 3-D scenes (lidar-like): per cloud a size uniform
    in [n_min, n_max]; (1 - ground_frac) of its points from 5..60 Gaussian
    blobs (std uniform in [sigma_lo, sigma_hi] m, centres uniform in the box),
    the rest a ground layer with x, y uniform over the box and z ~ N(0,
    ground_sigma^2).  Rows are padded with zeros to ``pad_to`` floats so each
    point starts on a 16-byte boundary.

    Returns ``(x [total, pad_to] float32, offsets int64[n_clouds + 1])``."""
    rng = _rng(seed)
    sizes = rng.integers(n_min, n_max + 1, size=n_clouds)
    offsets = np.zeros(n_clouds + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    x = np.zeros((total, pad_to), dtype=np.float32)
    bx = np.asarray(box, dtype=np.float64)
    for b in range(n_clouds):
        nb = int(sizes[b])
        n_ground = int(round(ground_frac * nb))
        n_blob = nb - n_ground
        k = int(rng.integers(blobs_min, blobs_max + 1))
        cen = rng.uniform(0.0, 1.0, size=(k, 3)) * bx
        sig = rng.uniform(sigma_lo, sigma_hi, size=k)
        which = rng.integers(0, k, size=n_blob)
        pts = cen[which] + sig[which, None] * rng.standard_normal((n_blob, 3))
        g = np.empty((n_ground, 3))
        g[:, 0] = rng.uniform(0.0, bx[0], size=n_ground)
        g[:, 1] = rng.uniform(0.0, bx[1], size=n_ground)
        g[:, 2] = ground_sigma * rng.standard_normal(n_ground)
        cloud = np.concatenate([pts, g])[rng.permutation(nb)]
        x[offsets[b]:offsets[b + 1], :3] = cloud
    return x, offsets


def random_points(n: int, d: int, seed: int, kind: str = "mixture") -> np.ndarray:
    """Small test inputs.  ``mixture``: a few tight Gaussian blobs in [0,1]^d
    plus uniform noise; ``grid``: small integers (exact in FP32, so FP32 and
    FP64 squared distances agree exactly); ``uniform``: uniform on [0,1]^d."""
    rng = _rng(seed)
    if kind == "grid":
        return rng.integers(0, 6, size=(n, d)).astype(np.float32)
    if kind == "uniform":
        return rng.uniform(0.0, 1.0, size=(n, d)).astype(np.float32)
    k = max(1, min(6, n // 20))
    c = rng.uniform(0.0, 1.0, size=(k, d))
    which = rng.integers(0, k, size=n)
    x = c[which] + (0.05 / math.sqrt(d)) * rng.standard_normal((n, d))
    noise = rng.uniform(0.0, 1.0, size=n) < 0.1
    x[noise] = rng.uniform(0.0, 1.0, size=(int(noise.sum()), d))
    return np.ascontiguousarray(x.astype(np.float32))


def eps_quantile(x: np.ndarray, q: float = 0.01, n_pairs: int = 1_000_000, seed: int = 0) -> float:
    """eps as the q-quantile of Euclidean distances over n_pairs seeded random
    pairs (i != j, PCG64), nearest rank: the ceil(q * n_pairs)-th smallest FP64
    distance, returned as float32."""
    rng = _rng(seed ^ 0xE95)
    n = x.shape[0]
    i = rng.integers(0, n, size=n_pairs)
    j = rng.integers(0, n - 1, size=n_pairs)
    j = j + (j >= i)
    d2 = np.empty(n_pairs, dtype=np.float64)
    chunk = 1 << 16
    for s in range(0, n_pairs, chunk):
        e = min(n_pairs, s + chunk)
        diff = x[i[s:e]].astype(np.float64) - x[j[s:e]].astype(np.float64)
        d2[s:e] = np.einsum("ij,ij->i", diff, diff)
    k = max(1, int(math.ceil(q * n_pairs)))
    kth = np.partition(d2, k - 1)[k - 1]
    return float(np.float32(math.sqrt(kth)))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as the uint16 bit patterns.  Non-finite inputs keep their class."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u.astype(np.uint64) + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x)
    if nan.any():
        r[nan] = 0x7FC0
    return r


def bf16_to_f32(b: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns (uint16) to float32 values."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def mlp_init(d_in: int, hidden: int, seed: int) -> dict:
    """Initial surrogate weights (uniform +-1/sqrt(fan_in), the usual default
    for linear layers), float32."""
    rng = _rng(seed)

    def u(shape, fan_in):
        b = 1.0 / math.sqrt(fan_in)
        return rng.uniform(-b, b, size=shape).astype(np.float32)

    return dict(w1=u((hidden, d_in), d_in), b1=u((hidden,), d_in),
                w2=u((hidden, hidden), hidden), b2=u((hidden,), hidden),
                w3=u((hidden,), hidden), b3=u((1,), hidden))
