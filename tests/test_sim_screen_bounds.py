"""The certificate of the tensor-core screens' similarity form (inner
product and cosine, over the BF16 or the FP8 copy), checked on the CPU in
exact arithmetic on emulated copy and FP32 values: the copy kernels' squared
norms and error bounds, the MMA's dot product anywhere within its allowance
of the exact one, then the device's interval arithmetic for <a,b> (and, for
cosine, its division by the interval of |a| |b|) in FP32 with IEEE
roundings.  Every pair kept must have a similarity strictly above tau +
band and every pair dropped one strictly below tau - band: decided as the
FP64 oracle decides, and never one of the reported band."""
from fractions import Fraction

import numpy as np
import pytest

from test_mma_screen_bounds import MMA_REL, bf16, e4m3, f32, fma32, fp8_scale, row_data

SIM_CM = {"bf16": 2.0 ** -17, "fp8": 2.0 ** -11}


def round_up32(v):
    f = np.float32(float(v))
    while Fraction(float(f)) < v:
        f = np.nextafter(f, np.float32(np.inf))
    return f


def round_down32(v):
    f = np.float32(float(v))
    while Fraction(float(f)) > v:
        f = np.nextafter(f, np.float32(-np.inf))
    return f


def decide(dot, na2, ea, nb2, eb, cosine, cm, keep_thr, drop_thr):
    """The device's decision in FP32: 1 keep, 0 drop, -1 open."""
    p12 = np.float32(1 + 2.0 ** -12)
    ra, rb = np.sqrt(na2), np.sqrt(nb2)            # correctly rounded
    na, nb = np.float32(ra * p12), np.float32(rb * p12)
    eta = fma32(ea, np.float32(nb + eb), np.float32(na * eb))
    eta = fma32(np.float32(np.float32(np.float32(cm) + np.float32(2.0 ** -24)) * na), nb, eta)
    eta = np.float32(fma32(eta, np.float32(2.0 ** -20), eta) + np.float32(2.0 ** -100))
    w = np.float32(np.float32(2.0 ** -22) * np.float32(abs(dot)))
    lo = np.float32(np.float32(dot - eta) - w)
    hi = np.float32(np.float32(dot + eta) + w)
    if cosine:
        al = np.float32(fma32(ra, np.float32(-(2.0 ** -12)), ra) - ea)
        bl = np.float32(fma32(rb, np.float32(-(2.0 ** -12)), rb) - eb)
        ah, bh = np.float32(na + ea), np.float32(nb + eb)
        if not (al >= 2.0 ** -60 and bl >= 2.0 ** -60 and ah <= 2.0 ** 60 and bh <= 2.0 ** 60):
            return -1
        pl = np.float32(np.float32(al * bl) * np.float32(1 - 2.0 ** -22))
        ph = np.float32(np.float32(ah * bh) * np.float32(1 + 2.0 ** -22))
        cl = np.float32(lo / ph) if lo >= 0 else np.float32(lo / pl)
        ch = np.float32(hi / pl) if hi >= 0 else np.float32(hi / ph)
        lo = np.float32(cl - np.float32(np.float32(2.0 ** -22) * np.float32(abs(cl))))
        hi = np.float32(ch + np.float32(np.float32(2.0 ** -22) * np.float32(abs(ch))))
    if lo >= keep_thr:
        return 1
    if hi < drop_thr:
        return 0
    return -1


def cos_cmp(dot, na2, nb2, t):
    """sign of (dot / sqrt(na2 nb2) - t), exactly."""
    if dot >= 0 > t:
        return 1
    if dot < 0 <= t:
        return -1
    lhs, rhs = dot * dot, t * t * na2 * nb2
    if dot >= 0:
        return (lhs > rhs) - (lhs < rhs)
    return (lhs < rhs) - (lhs > rhs)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("exact_copy", [False, True])
@pytest.mark.parametrize("cosine", [False, True])
@pytest.mark.parametrize("d", [8, 64, 128])
def test_similarity_screen_decides_only_outside_the_band(d, cosine, exact_copy, kind):
    """exact_copy: points the copy holds exactly and a band of 10^-8, so
    that only the MMA allowance stands between a decision and the band."""
    rng = np.random.default_rng(3 * d + cosine + 5 * exact_copy + 17 * (kind == "fp8"))
    band_rel = 1e-8 if exact_copy else 1e-5
    n_rows = 40
    rows = [(rng.standard_normal(d) * np.float32(2.0 ** rng.integers(-2, 3))).astype(np.float32)
            for _ in range(n_rows)]
    if cosine:
        rows = [(r / np.float32(np.linalg.norm(r))).astype(np.float32) for r in rows]
    pairs = []
    for _ in range(250):
        ia = int(rng.integers(0, n_rows))
        b = (rows[ia] + rng.standard_normal(d) * float(rng.uniform(0.05, 1.5))
             * float(np.linalg.norm(rows[ia])) / np.sqrt(d)).astype(np.float32)
        if cosine:
            b = (b / np.float32(np.linalg.norm(b))).astype(np.float32)
        pairs.append((ia, b))
    k = 0
    if kind == "fp8":
        k = fp8_scale(max(float(np.max(np.abs(v))) for v in rows + [b for _, b in pairs]))
    if exact_copy:
        def hold(v):
            if kind == "bf16":
                return bf16(v)
            return (e4m3((v * np.float32(2.0 ** k)).astype(np.float32))
                    * 2.0 ** -k).astype(np.float32)
        rows = [hold(v) for v in rows]
        pairs = [(ia, hold(b)) for ia, b in pairs]
    data = [row_data(v, kind, k) for v in rows]
    decided = 0
    for t, (ia, b) in enumerate(pairs):
        a = rows[ia]
        sa, _, na2, ea = data[ia]
        sb, _, nb2, eb = row_data(b, kind, k)
        fa = [Fraction(float(v)) for v in a]
        fb = [Fraction(float(v)) for v in b]
        dot_x = sum(u * v for u, v in zip(fa, fb))
        n2a, n2b = sum(u * u for u in fa), sum(v * v for v in fb)
        # tau near the pair's own similarity, some within the band
        sim = float(dot_x) / (float(n2a) * float(n2b)) ** 0.5 if cosine else float(dot_x)
        rel = rng.choice([0.0, 3e-7, -3e-7, 3e-6, -3e-6, 3e-5, -3e-5, 1e-3, -1e-3, 0.02, -0.02,
                          0.2, -0.2])
        tau = np.float32(sim - rel * max(abs(sim), 1e-3))
        band = Fraction(band_rel) * abs(Fraction(float(tau)))
        bw = band * (1 + Fraction(1, 2 ** 20))
        keep_thr = round_up32(Fraction(float(tau)) + bw)
        drop_thr = round_down32(Fraction(float(tau)) - bw)
        scale = Fraction(2) ** (-2 * k)
        dab = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(sa, sb))
        mag = sum(abs(Fraction(float(u)) * Fraction(float(v))) for u, v in zip(sa, sb))
        for sgn in (-1, 0, 1):
            dot = f32((dab + sgn * MMA_REL[kind] * mag)) if kind == "bf16" else \
                np.float32(f32(dab + sgn * MMA_REL[kind] * mag) * np.float32(float(scale)))
            dec = decide(dot, na2, ea, nb2, eb, cosine, SIM_CM[kind], keep_thr, drop_thr)
            if dec < 0:
                continue
            decided += 1
            hi_t, lo_t = Fraction(float(tau)) + band, Fraction(float(tau)) - band
            if cosine:
                if dec == 1:
                    assert cos_cmp(dot_x, n2a, n2b, hi_t) > 0, (kind, d, t, sgn, rel)
                else:
                    assert cos_cmp(dot_x, n2a, n2b, lo_t) < 0, (kind, d, t, sgn, rel)
            else:
                if dec == 1:
                    assert dot_x > hi_t, (kind, d, t, sgn, rel)
                else:
                    assert dot_x < lo_t, (kind, d, t, sgn, rel)
    assert decided > 60, decided
