"""The certificate of the tensor-core screens -- over the BF16 copy (the
headline's gather) and over the FP8 (E4M3) copy of x 2^k -- checked on the
CPU in exact rational arithmetic on emulated BF16 / E4M3 / FP32 values: the
copy of each row, its norm bound, the squared norm of the copy and the
copy's error bound as the copy kernels form them; the MMA's dot product of
the copies anywhere within 2^-17 (BF16) or 2^-11 (E4M3) of sum |a'_k b'_k|
around the exact one (the allowances the screens assume for the tensor
cores' accumulation);
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
# evaluation allowance of d2 per (|a| + |b|)^2, and the MMA's accumulation
# allowance per sum |a'_k b'_k|, for each copy
C_ABS = {"bf16": 2.0 ** -15, "fp8": 2.0 ** -9}
MMA_REL = {"bf16": Fraction(1, 2 ** 17), "fp8": Fraction(1, 2 ** 11)}


def e4m3(v):
    """Round values to E4M3 (3 fraction bits, normal exponents from -6,
    subnormal steps of 2^-9, saturating at 448), ties to even."""
    out = np.empty(len(v), dtype=np.float64)
    for t, x in enumerate(v):
        a = abs(Fraction(float(x)))
        if a == 0:
            out[t] = 0.0
            continue
        e = max(math.floor(math.log2(a)), -6)
        while Fraction(2) ** e > a:
            e -= 1
        while Fraction(2) ** (e + 1) <= a:
            e += 1
        e = max(e, -6)
        step = Fraction(2) ** (e - 3)
        r = min(round(a / step) * step, Fraction(448))
        out[t] = float(r) * (1 if x >= 0 else -1)
    return out


def fp8_scale(amax):
    m, e = math.frexp(float(amax))
    return max(-60, min(60, 8 - e)) if amax > 0 else 0


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


def row_data(x, kind, k=0):
    """Copy of x (in the units of x), norm bound of x, squared norm of the
    copy and the copy's error bound, as the copy kernels form them."""
    nrm = f32(f32(math.sqrt(float(fsum_fma(x)))) * np.float32(1 + 2.0 ** -11))
    if kind == "bf16":
        xb = bf16(x)
        stored = xb
        nb2 = fsum_fma(xb)          # squares of BF16 values are exact in FP32
        diff = (x - xb).astype(np.float32)
    else:
        q = e4m3((x * np.float32(2.0 ** k)).astype(np.float32)).astype(np.float32)
        stored = q
        xb = (q * np.float32(2.0 ** -k)).astype(np.float32)
        nb2 = f32(float(fsum_fma(q)) * 2.0 ** (-2 * k))
        diff = np.array([f32(float(u) - float(w)) for u, w in zip(x, xb)], dtype=np.float32)
    se = fsum_fma(diff)
    err = fma32(f32(math.sqrt(float(se))), np.float32(1 + 2.0 ** -11), np.float32(2.0 ** -60))
    return stored, nrm, nb2, err


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


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("exact_copy", [False, True])
@pytest.mark.parametrize("d", [5, 16, 32, 64, 100, 128])
def test_tensor_core_screen_decides_only_outside_the_band(d, exact_copy, kind):
    """exact_copy: points that the copy holds exactly, so its error bounds
    are 2^-60 and only the MMA and evaluation allowances stand between a
    decision and the band."""
    rng = np.random.default_rng(1000 + d + 7 * exact_copy + 13 * (kind == "fp8"))
    band_rel = 1e-5
    rows = []
    for _ in range(40 if kind == "fp8" else 60):
        scale = np.float32(2.0 ** rng.integers(-3, 4))
        rows.append((rng.standard_normal(d) * scale).astype(np.float32))
    pairs = []
    for _ in range(300):
        ia = int(rng.integers(0, len(rows)))
        direction = rng.standard_normal(d)
        direction /= np.linalg.norm(direction)
        r = float(np.linalg.norm(rows[ia])) * float(rng.uniform(*((0.05, 0.6) if kind == "bf16"
                                                                   else (0.3, 1.2))))
        pairs.append((ia, (rows[ia] + direction * r).astype(np.float32)))
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
    nrm_max = max(dd[1] for dd in data + [row_data(b, kind, k) for _, b in pairs])
    err_max = max(dd[3] for dd in data + [row_data(b, kind, k) for _, b in pairs])
    # the MMA's dot product is in the units of the stored values:
    # d2 = fma(-2^(1 - 2k), dot, |a'|^2 + |b'|^2)
    m2inv = np.float32(-(2.0 ** (1 - 2 * k)))
    decided = kept = 0
    for t, (ia, b) in enumerate(pairs):
        a = rows[ia]
        sa, nrm_a, na2, ea = data[ia]
        sb, nrm_b, nb2, eb = row_data(b, kind, k)
        exact = sum((Fraction(float(u)) - Fraction(float(v))) ** 2 for u, v in zip(a, b))
        rel = rng.choice([0.0, 3e-6, -3e-6, 1e-5, -1e-5, 3e-5, -3e-5, 1e-4, -1e-4, 3e-3, -3e-3,
                          0.05, -0.05, 0.2, -0.2] + ([0.5, -0.5, 1.0, -0.7] if kind == "fp8" else []))
        eps = np.float32(math.sqrt(float(exact)) * (1 + rel))
        lo_eps, hi_eps, g = host_constants(eps, band_rel, d)
        dot_exact = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(sa, sb))
        mag = sum(abs(Fraction(float(u)) * Fraction(float(v))) for u, v in zip(sa, sb))
        nsum = f32(float(nrm_a) + float(nrm_max))
        e_abs = fma32(f32(C_ABS[kind] * float(nsum)), nsum, np.float32(2.0 ** -100))
        keep_row, drop_row = thresholds(lo_eps, hi_eps, g, f32(float(ea) + float(err_max)), e_abs)
        eps2 = Fraction(float(eps)) ** 2
        for sgn in (-1, 0, 1):
            dot = f32(dot_exact + sgn * MMA_REL[kind] * mag)
            d2 = fma32(m2inv, dot, f32(float(na2) + float(nb2)))
            keep = d2 <= keep_row
            open_ = not keep and not d2 > drop_row
            if open_:
                kt, dt = thresholds(lo_eps, hi_eps, g, f32(float(ea) + float(eb)), e_abs)
                keep = d2 <= kt
                open_ = not keep and not d2 > dt
            if keep:
                decided += 1
                kept += 1
                assert exact < eps2 * (1 - Fraction(band_rel)), (kind, d, t, sgn, rel)
            elif not open_:
                decided += 1
                assert exact > eps2 * (1 + Fraction(band_rel)), (kind, d, t, sgn, rel)
    assert decided > 60 and kept > 30, (decided, kept)


def _group_sum(ab, bb, lanes, vec):
    """FP32 sum of (a'_k - b'_k)^2 with element k on lane (k // vec) % lanes,
    fused multiply-adds in order per lane, then a pairwise tree."""
    acc = [np.float32(0.0)] * lanes
    for k in range(ab.size):
        t = np.float32(ab[k] - bb[k])
        lane = (k // vec) % lanes
        acc[lane] = fma32(t, t, acc[lane])
    while len(acc) > 1:
        acc = [np.float32(acc[2 * i] + acc[2 * i + 1]) for i in range(len(acc) // 2)]
    return acc[0]


@pytest.mark.parametrize("exact_copy", [False, True])
@pytest.mark.parametrize("d", [5, 16, 64, 130])
def test_cuda_core_screen_decides_only_outside_the_band(d, exact_copy):
    """The screen on CUDA cores: eta = 2^-8 (|a| + |b|) + 2^-60 from the
    rows' norm bounds, the FP32 sum over the copy in the group order of the
    BF16 mapping (8-value chunks, lanes a power of two), thresholds
    (eps sqrt(1 -+ band_rel) -+ eta)^2 (1 -+ g); partner bound its own or the
    largest of the set."""
    rng = np.random.default_rng(300 + d + exact_copy)
    band_rel = 1e-8 if exact_copy else 1e-5
    chunks = -(-d // 8)
    lanes = 1
    while lanes < chunks and lanes < 32:
        lanes <<= 1
    screen_u = np.float32(2.0 ** -8 * (1 + 2.0 ** -20))
    rows = [(rng.standard_normal(d) * np.float32(2.0 ** rng.integers(-3, 4))).astype(np.float32)
            for _ in range(40)]
    if exact_copy:
        rows = [bf16(r) for r in rows]
    nrms = [row_data(r, "bf16")[1] for r in rows]
    nrm_max = max(nrms)
    decided = 0
    for t in range(250):
        ia = int(rng.integers(0, len(rows)))
        a = rows[ia]
        direction = rng.standard_normal(d)
        direction /= np.linalg.norm(direction)
        b = (a + direction * float(np.linalg.norm(a)) * float(rng.uniform(0.05, 0.8))
             ).astype(np.float32)
        if exact_copy:
            b = bf16(b)
        nrm_b = row_data(b, "bf16")[1]
        exact = sum((Fraction(float(u)) - Fraction(float(v))) ** 2 for u, v in zip(a, b))
        rel = rng.choice([0.0, 3e-6, -3e-6, 1e-5, -1e-5, 1e-3, -1e-3, 0.02, -0.02, 0.1, -0.1])
        eps = np.float32(math.sqrt(float(exact)) * (1 + rel))
        lo_eps, hi_eps, g = host_constants(eps, band_rel, d)
        s = _group_sum(bf16(a), bf16(b), lanes, 8)
        for nrm_p in (nrm_b, nrm_max):
            eta = fma32(screen_u, np.float32(nrms[ia] + nrm_p), np.float32(2.0 ** -60))
            lo = np.float32(lo_eps - eta)
            hi = np.float32(hi_eps + eta)
            keep_thr = np.float32(np.float32(lo * lo) * np.float32(1 - g)) \
                if lo > np.float32(2.0 ** -10) * lo_eps else np.float32(-1.0)
            drop_thr = np.float32(np.float32(hi * hi) * np.float32(1 + g))
            eps2 = Fraction(float(eps)) ** 2
            if s <= keep_thr:
                decided += 1
                assert exact < eps2 * (1 - Fraction(band_rel)), (d, t, rel)
            elif s > drop_thr:
                decided += 1
                assert exact > eps2 * (1 + Fraction(band_rel)), (d, t, rel)
    assert decided > 60, decided
