"""The certified band of the plain similarity gather (inner product and
cosine over FP32 points), checked on the CPU in exact arithmetic on
emulated FP32 values: the dot product and the partner's squared norm by
fused multiply-adds per lane and a pairwise tree over the group, the
source's squared norm the same way, rsqrtf anywhere within its documented 2
ulp, and the kernel's decision -- keep at sim - err >= tau, drop at sim +
err < tau, err = c1 |a| |b| (+ band) for the inner product or c1 + c2 |cos|
(+ band) for cosine, c1 = 2 (K + L + 3) u + 2^-22 and c2 = 2 (2 e_inv + 3u),
e_inv = (K_n / 2 + 5) u.  Every kept pair must lie strictly above tau +
band and every dropped one strictly below tau - band."""
import math
from fractions import Fraction

import numpy as np
import pytest

from test_mma_screen_bounds import fma32
from test_sim_screen_bounds import cos_cmp, round_up32

U = 2.0 ** -24


def group_sums(a, b, lanes, vec):
    """(dot, |b|^2) in FP32 in the group order; K = terms per lane."""
    dot = [np.float32(0.0)] * lanes
    nb = [np.float32(0.0)] * lanes
    cnt = [0] * lanes
    for k in range(a.size):
        lane = (k // vec) % lanes
        dot[lane] = fma32(a[k], b[k], dot[lane])
        nb[lane] = fma32(b[k], b[k], nb[lane])
        cnt[lane] += 1
    levels = 0
    while len(dot) > 1:
        dot = [np.float32(dot[2 * i] + dot[2 * i + 1]) for i in range(len(dot) // 2)]
        nb = [np.float32(nb[2 * i] + nb[2 * i + 1]) for i in range(len(nb) // 2)]
        levels += 1
    return dot[0], nb[0], max(cnt), levels


def rsqrt_ulps(v, k):
    """1/sqrt(v) correctly rounded, then moved by k ulps (k in -2..2)."""
    r = np.float32(1.0 / math.sqrt(float(v)))
    step = np.float32(np.inf) if k > 0 else np.float32(0)
    for _ in range(abs(k)):
        r = np.nextafter(r, step)
    return r


@pytest.mark.parametrize("tight", [False, True])
@pytest.mark.parametrize("cosine", [False, True])
@pytest.mark.parametrize("layout", [(1, 4), (4, 4), (8, 4), (16, 4)])
@pytest.mark.parametrize("d", [4, 16, 64, 128])
def test_similarity_band_certifies_every_decision(d, layout, cosine, tight):
    """tight: band 10^-9 and near-ties within 10^-7, so c1 and c2 alone
    stand between a decision and tau."""
    lanes, vec = layout
    rng = np.random.default_rng(d + 11 * lanes + 3 * cosine + tight)
    band_rel = 1e-9 if tight else 1e-5
    decided = 0
    for t in range(120):
        a = (rng.standard_normal(d) * np.float32(2.0 ** rng.integers(-4, 5))).astype(np.float32)
        b = (a * np.float32(rng.uniform(-1, 1)) + rng.standard_normal(d).astype(np.float32)
             * np.float32(rng.uniform(0.05, 2.0)) * np.float32(np.linalg.norm(a) / math.sqrt(d))
             ).astype(np.float32)
        dot, bb, fmas, levels = group_sums(a, b, lanes, vec)
        _, nn, _, _ = group_sums(a, a, lanes, vec)
        fa = [Fraction(float(v)) for v in a]
        fb = [Fraction(float(v)) for v in b]
        dot_x = sum(u * v for u, v in zip(fa, fb))
        n2a, n2b = sum(u * u for u in fa), sum(v * v for v in fb)
        sim = float(dot_x) / math.sqrt(float(n2a) * float(n2b)) if cosine else float(dot_x)
        rel = rng.choice([0.0, 1e-7, -1e-7, 1e-6, -1e-6, 1e-5, -1e-5, 1e-3, -1e-3, 0.05, -0.05]
                         if tight else [0.0, 3e-6, -3e-6, 3e-5, -3e-5, 1e-3, -1e-3, 0.05, -0.05])
        tau = np.float32(sim - rel * max(abs(sim), 1e-3))
        band = Fraction(band_rel) * abs(Fraction(float(tau)))
        band_f = round_up32(band)
        c1 = round_up32(Fraction(2 * (fmas + levels + 3)) * Fraction(U) + Fraction(2) ** -22)
        e_inv = (Fraction(fmas + levels, 2) + 5) * Fraction(U)
        c2 = round_up32(2 * (2 * e_inv + 3 * Fraction(U))) if cosine else np.float32(0)
        for ka in (-2, 0, 2):
            for kb in (-2, 0, 2):
                r = rsqrt_ulps(nn, ka)
                scale_i = r if cosine else np.float32(nn * r)
                inv_p = rsqrt_ulps(bb, kb)
                if cosine:
                    s32 = np.float32(np.float32(dot * scale_i) * inv_p)
                    err = np.float32(c1 + np.float32(c2 * np.float32(abs(s32))))
                else:
                    s32 = dot
                    err = np.float32(c1 * np.float32(scale_i * np.float32(bb * inv_p)))
                err = np.float32(err + band_f)
                lo_t, hi_t = Fraction(float(tau)) - band, Fraction(float(tau)) + band
                if np.float32(s32 - err) >= tau:
                    decided += 1
                    ok = cos_cmp(dot_x, n2a, n2b, hi_t) > 0 if cosine else dot_x > hi_t
                    assert ok, (d, lanes, t, ka, kb, rel)
                elif np.float32(s32 + err) < tau:
                    decided += 1
                    ok = cos_cmp(dot_x, n2a, n2b, lo_t) < 0 if cosine else dot_x < lo_t
                    assert ok, (d, lanes, t, ka, kb, rel)
    assert decided > 300, decided
