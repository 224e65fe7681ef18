"""The guard band of the FP32 squared distance (the plain gather's, the
sequential recheck order's and the queue kernel's warp-wide order), checked
on the CPU in exact arithmetic: with K fused multiply-adds per lane and L
levels of a pairwise tree, the FP32 value is within (K + L + 3) u relative
of the exact sum of squared differences, so a pair with d2 below
eps^2 (1 - (band_rel + delta)) or above eps^2 (1 + (band_rel + delta)),
delta = 2 (K + L + 3) u + 2^-22 (thresholds rounded outwards), lies strictly
inside or outside the reported band: decided as the FP64 oracle decides.
Rows span many binades; partners are planted at distances near eps."""
import math
from fractions import Fraction

import numpy as np
import pytest

from test_mma_screen_bounds import fma32

U = 2.0 ** -24


def guard(eps2, band_rel, fmas, levels):
    """The library's thresholds: eps2 (1 -+ (band_rel + delta)), outwards."""
    delta = 2.0 * (fmas + levels + 3) * U + 2.0 ** -22
    lo = Fraction(eps2) * (1 - Fraction(float(np.float32(band_rel))) - Fraction(delta))
    hi = Fraction(eps2) * (1 + Fraction(float(np.float32(band_rel))) + Fraction(delta))
    lof, hif = np.float32(float(lo)), np.float32(float(hi))
    while Fraction(float(lof)) > lo:
        lof = np.nextafter(lof, np.float32(0))
    while Fraction(float(hif)) < hi:
        hif = np.nextafter(hif, np.float32(np.inf))
    return lof, hif


def lanes_value(a, b, lanes, vec):
    """FP32 d2 with element k on lane (k // vec) % lanes, each lane's
    differences squared and added by fused multiply-adds in order, then a
    pairwise tree over the lanes.  Returns (d2, K, L)."""
    acc = [np.float32(0.0)] * lanes
    count = [0] * lanes
    for k in range(a.size):
        lane = (k // vec) % lanes
        t = np.float32(a[k] - b[k])
        acc[lane] = fma32(t, t, acc[lane])
        count[lane] += 1
    levels = 0
    while len(acc) > 1:
        acc = [np.float32(acc[2 * i] + acc[2 * i + 1]) for i in range(len(acc) // 2)]
        levels += 1
    return acc[0], max(count), levels


@pytest.mark.parametrize("layout", [("sequential", 1, 1), ("group4", 4, 4), ("group8", 8, 4),
                                    ("group16", 16, 4), ("warp", 32, 1)])
@pytest.mark.parametrize("band_rel", [1e-5, 0.0])
@pytest.mark.parametrize("d", [1, 3, 16, 64, 130])
def test_fp32_guard_band_certifies_every_decision(d, layout, band_rel):
    """band_rel = 0 with partners within 10^-7 of eps: only delta stands
    between a decision and eps itself."""
    _, lanes, vec = layout
    rng = np.random.default_rng(d * 7 + lanes + int(band_rel == 0))
    decided = 0
    for t in range(300):
        scale = np.exp2(rng.integers(-20, 21, d)).astype(np.float32)
        a = (rng.standard_normal(d) * scale).astype(np.float32)
        b = (a + rng.standard_normal(d).astype(np.float32) * np.float32(rng.uniform(0.01, 2))
             * np.float32(np.linalg.norm(a) / math.sqrt(d))).astype(np.float32)
        exact = sum((Fraction(float(u)) - Fraction(float(v))) ** 2 for u, v in zip(a, b))
        if exact == 0:
            continue
        d2, fmas, levels = lanes_value(a, b, lanes, vec)
        # the relative bound itself
        assert abs(Fraction(float(d2)) - exact) <= (fmas + levels + 3) * Fraction(U) * exact
        rel = rng.choice([0.0, 3e-6, -3e-6, 1e-5, -1e-5, 3e-5, -3e-5, 1e-4, -1e-4, 0.01, -0.01]
                         if band_rel else [5e-8, -5e-8, 1e-7, -1e-7, 3e-7, -3e-7, 1e-6, -1e-6,
                                           1e-5, -1e-5, 1e-4, -1e-4])
        eps = np.float32(math.sqrt(float(exact)) * (1 + rel))
        eps2 = Fraction(float(eps)) ** 2
        lo, hi = guard(float(eps2), band_rel, fmas, levels)
        if d2 < lo:
            decided += 1
            assert exact < eps2 * (1 - Fraction(band_rel)), (d, t, rel)
        elif d2 > hi:
            decided += 1
            assert exact > eps2 * (1 + Fraction(band_rel)), (d, t, rel)
    assert decided > 80, decided
