"""The error analysis behind the BF16 screen of the Manhattan and Chebyshev
distances, checked on the CPU with exact arithmetic: (1) the rounding of a
row to BF16 moves it by at most sqrt(d) e2 in L1 and e2 in L-inf, e2 the
Euclidean bound the copy carries (its FP32 sum of squared differences times
1 + 2^-11, plus 2^-60); (2) the FP32 value over two copied rows in the
kernel's order (differences rounded once, two terms per 16-byte chunk into
each of four partials, pairwise combination, two shuffle levels) is within
c'' = (2 ceil(chunks / 4) + 5) u of the exact L1 distance of the copies and
within u of their L-inf distance; (3) with those, the keep / drop
thresholds eps (1 -+ (band_rel + c)) -+ eta put every decided pair strictly
inside or outside eps (1 -+ band_rel), so none of the reported band is
decided on the copy.  Inputs span many binades, with planted near-ties."""
import math
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -24


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def copy_error_bound(x):
    """The copy's Euclidean error bound as the library forms it: FP32 sum of
    squared differences (exact differences), sqrt, times 1 + 2^-11, + 2^-60."""
    e = (x - bf16(x)).astype(np.float32)
    se = np.float32(0.0)
    for v in e:                     # any FP32 order: within (d + 6) u of exact
        se = np.float32(se + np.float32(v * v))
    return float(np.float32(np.float32(math.sqrt(float(se))) * np.float32(1 + 2.0 ** -11))) \
        + 2.0 ** -60


def kernel_order(a, b, linf):
    """FP32 distance of two copied rows in the screened kernel's order."""
    d = a.size
    ld = -(-d // 8) * 8
    aa = np.zeros(ld, np.float32)
    bb = np.zeros(ld, np.float32)
    aa[:d], bb[:d] = a, b
    nc = ld // 8

    def comb(x, y):
        return np.float32(max(x, y)) if linf else np.float32(x + y)

    lanes = []
    for q in range(4):
        acc = [np.float32(0.0)] * 4
        for c in range(q, nc, 4):
            for e in range(8):
                k = 8 * c + e
                t = np.float32(abs(np.float32(aa[k] - bb[k])))
                acc[e & 3] = comb(acc[e & 3], t)
        lanes.append(comb(comb(acc[0], acc[1]), comb(acc[2], acc[3])))
    v01, v23 = comb(lanes[0], lanes[1]), comb(lanes[2], lanes[3])
    return float(comb(v01, v23)), nc


def exact_l1(a, b):
    return sum(abs(Fraction(float(x)) - Fraction(float(y))) for x, y in zip(a, b))


def exact_linf(a, b):
    return max(abs(Fraction(float(x)) - Fraction(float(y))) for x, y in zip(a, b))


def _rows(rng, d, spread):
    scale = np.exp2(rng.integers(-spread, spread + 1, d)).astype(np.float32)
    return (rng.standard_normal(d).astype(np.float32) * scale).astype(np.float32)


@pytest.mark.parametrize("d", [1, 3, 8, 31, 64, 65, 128, 200])
def test_copy_error_bounds_in_l1_and_linf(d):
    rng = np.random.default_rng(d)
    for _ in range(60):
        x = _rows(rng, d, 12)
        xb = bf16(x)
        e2 = Fraction(copy_error_bound(x))
        l1 = sum(abs(Fraction(float(u)) - Fraction(float(v))) for u, v in zip(x, xb))
        li = max(abs(Fraction(float(u)) - Fraction(float(v))) for u, v in zip(x, xb))
        # sqrt(d) rounded up as the library's factor sqrt(d) (1 + 2^-10) is
        assert l1 <= Fraction(math.sqrt(d)) * (1 + Fraction(1, 1024)) * e2
        assert li <= e2


@pytest.mark.parametrize("d", [1, 4, 8, 33, 64, 128, 200])
@pytest.mark.parametrize("linf", [False, True])
def test_kernel_order_within_its_relative_bound(d, linf):
    rng = np.random.default_rng(100 + d + linf)
    worst = 0.0
    for _ in range(80):
        a = bf16(_rows(rng, d, 20))
        b = bf16(a + _rows(rng, d, 6) * np.float32(0.01)) if rng.random() < 0.5 \
            else bf16(_rows(rng, d, 20))
        v, nc = kernel_order(a, b, linf)
        ex = exact_linf(a, b) if linf else exact_l1(a, b)
        cpp = Fraction(U) if linf else (2 * (-(-nc // 4)) + 5) * Fraction(U)
        err = abs(Fraction(v) - ex)
        assert err <= cpp * ex, (d, float(err / ex) if ex else err)
        if ex:
            worst = max(worst, float(err / (cpp * ex)))
    assert worst <= 1.0


def _thresholds(eps, band_rel, d, ldb, linf):
    """The library's pm_lo / pm_hi / pm_escale in exact arithmetic (the
    FP32 roundings only move them outwards)."""
    nc = ldb // 8
    cpp = Fraction(U) if linf else (2 * (-(-nc // 4)) + 5) * Fraction(U)
    c = 2 * cpp + Fraction(2) ** -22
    lo = Fraction(eps) * (1 - Fraction(band_rel) - c)
    hi = Fraction(eps) * (1 + Fraction(band_rel) + c)
    scale = Fraction(1) if linf else Fraction(math.sqrt(d)) * (1 + Fraction(1, 1024))
    return lo, hi, scale, cpp


@pytest.mark.parametrize("d", [3, 16, 64, 130])
@pytest.mark.parametrize("linf", [False, True])
def test_decided_pairs_lie_outside_the_band(d, linf):
    rng = np.random.default_rng(7 * d + linf)
    band_rel = 1e-5
    ldb = -(-d // 8) * 8
    decided = 0
    for _ in range(200):
        a = _rows(rng, d, 3)
        # partners at distances near eps, some planted within the band
        b = (a + _rows(rng, d, 1) * np.float32(rng.uniform(0.2, 2.0))).astype(np.float32)
        ex = exact_linf(a, b) if linf else exact_l1(a, b)
        eps = float(np.float32(float(ex) * (1 + rng.choice([0.0, 3e-6, -3e-6, 1e-3, -1e-3,
                                                            0.05, -0.05, 0.3, -0.3]))))
        if eps <= 0:
            continue
        ea, eb = copy_error_bound(a), copy_error_bound(b)
        v, _ = kernel_order(bf16(a), bf16(b), linf)
        lo, hi, scale, _ = _thresholds(eps, band_rel, d, ldb, linf)
        eta = (Fraction(ea) + Fraction(eb)) * scale * (1 + Fraction(1, 1024))
        in_band = abs(ex - Fraction(eps)) <= Fraction(band_rel) * Fraction(eps)
        if Fraction(v) <= lo - eta:
            decided += 1
            assert ex < Fraction(eps) * (1 - Fraction(band_rel)) and not in_band
        elif Fraction(v) > hi + eta:
            decided += 1
            assert ex > Fraction(eps) * (1 + Fraction(band_rel)) and not in_band
    assert decided > 60, decided


def fp32_group_order(a, b, linf):
    """FP32 distance in the plain pair kernel's order over float4 chunks:
    lane q takes chunks q, q + 4, ...; one partial per vector component;
    (x + y) + (z + w); then two shuffle levels."""
    d = a.size
    nc = d // 4

    def comb(x, y):
        return np.float32(max(x, y)) if linf else np.float32(x + y)

    lanes = []
    for q in range(4):
        acc = [np.float32(0.0)] * 4
        for c in range(q, nc, 4):
            for e in range(4):
                k = 4 * c + e
                acc[e] = comb(acc[e], np.float32(abs(np.float32(a[k] - b[k]))))
        lanes.append(comb(comb(acc[0], acc[1]), comb(acc[2], acc[3])))
    return float(comb(comb(lanes[0], lanes[1]), comb(lanes[2], lanes[3])))


@pytest.mark.parametrize("band_rel", [1e-5, 0.0])
@pytest.mark.parametrize("linf", [False, True])
@pytest.mark.parametrize("d", [4, 8, 64, 128, 200])
def test_fp32_pair_guard_certifies_every_decision(d, linf, band_rel):
    """The plain pair kernel's guard band eps (1 -+ (band_rel + c)), c =
    2 (d + 2) u + 2^-22 for L1 and 4 u + 2^-22 for L-inf (rounded outwards):
    its FP32 value is within (d + 1) u (L1) or u (L-inf) of the exact
    distance, so every decision outside the band is the FP64 oracle's."""
    rng = np.random.default_rng(50 + d + 3 * linf + int(band_rel == 0))
    decided = 0
    for t in range(200):
        a = _rows(rng, d, 15)
        b = (a + _rows(rng, d, 2) * np.float32(rng.uniform(0.01, 1.0))).astype(np.float32)
        ex = exact_linf(a, b) if linf else exact_l1(a, b)
        if ex == 0:
            continue
        v = fp32_group_order(a, b, linf)
        assert abs(Fraction(v) - ex) <= (Fraction(U) if linf else (d + 1) * Fraction(U)) * ex
        rel = rng.choice([0.0, 5e-8, -5e-8, 3e-7, -3e-7, 3e-6, -3e-6, 1e-5, -1e-5, 1e-4, -1e-4,
                          0.01, -0.01])
        eps = np.float32(float(ex) * (1 + rel))
        c = (4 * Fraction(U) if linf else 2 * (d + 2) * Fraction(U)) + Fraction(2) ** -22
        lo = Fraction(float(eps)) * (1 - Fraction(float(np.float32(band_rel))) - c)
        hi = Fraction(float(eps)) * (1 + Fraction(float(np.float32(band_rel))) + c)
        if Fraction(v) < lo:
            decided += 1
            assert ex < Fraction(float(eps)) * (1 - Fraction(band_rel)), (d, t, rel)
        elif Fraction(v) > hi:
            decided += 1
            assert ex > Fraction(float(eps)) * (1 + Fraction(band_rel)), (d, t, rel)
    assert decided > 40, decided
