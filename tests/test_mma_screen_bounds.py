"""The certificate of the tensor-core BF16 screen (the headline's gather),
checked on the CPU in exact rational arithmetic on emulated BF16 / FP32
values: the copy of each row, its norm bound, the squared norm of the copy
and the copy's error bound as the copy kernel forms them; the MMA's dot
product of the copies anywhere within 2^-17 sum |a'_k b'_k| of the exact one
(the allowance the screen assumes for the tensor core's FP32 accumulation);
d2 = fma(-2, dot, |a'|^2 + |b'|^2) and the keep / drop thresholds in FP32 as
the kernel forms them (the row's against the largest partner bound, then
the pair's own).  Every pair it keeps must lie strictly inside eps sqrt(1 -
band_rel) and every pair it drops strictly outside eps sqrt(1 + band_rel):
decided exactly as the FP64 oracle decides, and never one of the reported
band.  Rows span several binades; partners are planted at distances near
eps, some inside the band."""
import math
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -24
C_ABS = 2.0 ** -15          # evaluation allowance of d2 per (|a| + |b|)^2
MMA_REL = Fraction(1, 2 ** 17)


def bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def f32(v):
    return np.float32(float(v))


def fma32(a, b, c):
    """FP32 fused multiply-add: the exact a b + c rounded once (through the
    correctly rounded double, whose second rounding is far inside the
    certificate's margins)."""
    return f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def fsum_fma(vals):
    s = np.float32(0.0)
    for v in vals:
        s = fma32(v, v, s)
    return s


def row_data(x):
    """Norm bound of x, squared norm of its copy, copy error bound."""
    xb = bf16(x)
    nrm = f32(f32(math.sqrt(float(fsum_fma(x)))) * np.float32(1 + 2.0 ** -11))
    nb2 = fsum_fma(xb)          # squares of BF16 values are exact in FP32
    se = fsum_fma((x - xb).astype(np.float32))
    err = fma32(f32(math.sqrt(float(se))), np.float32(1 + 2.0 ** -11), np.float32(2.0 ** -60))
    return xb, nrm, nb2, err


def host_constants(eps, band_rel, d):
    lo = Fraction(float(eps)) ** 2 * (1 - Fraction(band_rel))
    lo_eps = np.float32(math.sqrt(float(lo)))
    while Fraction(float(lo_eps)) ** 2 > lo:
        lo_eps = np.nextafter(lo_eps, np.float32(0))
    hi = Fraction(float(eps)) ** 2 * (1 + Fraction(band_rel))
    hi_eps = np.float32(math.sqrt(float(hi)))
    while Fraction(float(hi_eps)) ** 2 < hi:
        hi_eps = np.nextafter(hi_eps, np.float32(np.inf))
    chunks = -(-d // 8)
    group = 1
    while group < chunks and group < 32:
        group <<= 1
    nch, lg = -(-chunks // group), group.bit_length() - 1
    delta = 2.0 * (nch * 8 + lg + 3) * U + 2.0 ** -22
    g = np.float32(delta + 2.0 ** -20)
    if float(g) < delta + 2.0 ** -20:
        g = np.nextafter(g, np.float32(np.inf))
    return lo_eps, hi_eps, g


def thresholds(lo_eps, hi_eps, g, eta, e_abs):
    lo = f32(float(lo_eps) - float(eta))
    hi = f32(float(hi_eps) + float(eta))
    keep = fma32(f32(float(lo) * float(lo)), f32(1 - float(g)), -e_abs) \
        if lo > np.float32(2.0 ** -10) * lo_eps else np.float32(-1.0)
    drop = fma32(f32(float(hi) * float(hi)), f32(1 + float(g)), e_abs)
    return keep, drop


@pytest.mark.parametrize("exact_copy", [False, True])
@pytest.mark.parametrize("d", [5, 16, 32, 64, 100, 128])
def test_tensor_core_screen_decides_only_outside_the_band(d, exact_copy):
    """exact_copy: points that BF16 holds exactly, so the copy's error
    bounds are 2^-60 and only the MMA and evaluation allowances stand
    between a decision and the band."""
    rng = np.random.default_rng(1000 + d + 7 * exact_copy)
    band_rel = 1e-5
    rows = []
    for _ in range(60):
        scale = np.float32(2.0 ** rng.integers(-3, 4))
        r = (rng.standard_normal(d) * scale).astype(np.float32)
        rows.append(bf16(r) if exact_copy else r)
    data = [row_data(r) for r in rows]
    nrm_max = max(dd[1] for dd in data)
    err_max = max(dd[3] for dd in data)
    decided = kept = 0
    for k in range(400):
        ia = int(rng.integers(0, len(rows)))
        a = rows[ia]
        ab, nrm_a, na2, ea = data[ia]
        # a partner at a planted distance from a, eps near that distance
        direction = rng.standard_normal(d)
        direction /= np.linalg.norm(direction)
        r = float(np.linalg.norm(a)) * float(rng.uniform(0.05, 0.6))
        b = (a + direction * r).astype(np.float32)
        if exact_copy:
            b = bf16(b)
        bb, nrm_b, nb2, eb = row_data(b)
        exact = sum((Fraction(float(u)) - Fraction(float(v))) ** 2 for u, v in zip(a, b))
        rel = rng.choice([0.0, 3e-6, -3e-6, 1e-5, -1e-5, 3e-5, -3e-5, 1e-4, -1e-4, 3e-3, -3e-3,
                          0.05, -0.05, 0.2, -0.2])
        eps = np.float32(math.sqrt(float(exact)) * (1 + rel))
        lo_eps, hi_eps, g = host_constants(eps, band_rel, d)
        dot_exact = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(ab, bb))
        mag = sum(abs(Fraction(float(u)) * Fraction(float(v))) for u, v in zip(ab, bb))
        nsum = f32(float(nrm_a) + float(nrm_max))
        e_abs = fma32(f32(C_ABS * float(nsum)), nsum, np.float32(2.0 ** -100))
        keep_row, drop_row = thresholds(lo_eps, hi_eps, g, f32(float(ea) + float(err_max)), e_abs)
        eps2 = Fraction(float(eps)) ** 2
        for s in (-1, 0, 1):
            dot = f32(dot_exact + s * MMA_REL * mag)
            d2 = fma32(np.float32(-2.0), dot, f32(float(na2) + float(nb2)))
            keep = d2 <= keep_row
            open_ = not keep and not d2 > drop_row
            if open_:
                kt, dt = thresholds(lo_eps, hi_eps, g, f32(float(ea) + float(eb)), e_abs)
                keep = d2 <= kt
                open_ = not keep and not d2 > dt
            if keep:
                decided += 1
                kept += 1
                assert exact < eps2 * (1 - Fraction(band_rel)), (d, k, s, rel)
            elif not open_:
                decided += 1
                assert exact > eps2 * (1 + Fraction(band_rel)), (d, k, s, rel)
    assert decided > 150 and kept > 60, (decided, kept)
