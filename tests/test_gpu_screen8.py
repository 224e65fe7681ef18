"""The certified screen on an FP8 (E4M3) copy of FP32 points with tensor-core
dot products (SNG_FLAG_SCREEN8) against the FP64 oracle.  The copy's
rounding is coarse (2^-4 of the norms), so far more pairs stay open than with
the BF16 copy; the results must still be exactly the oracle's: CSR, degrees,
core flags and labels, for 64- and 128-byte rows, every register budget,
ragged draw counts and row ranges, every degree mode, the all-pairs draw,
rows far from the origin, exact ties at eps, tiny and huge scales (the copy's
power-of-two scale at both ends of its range), non-finite values, and the
1M-point workload at scale against the plain FP32 path."""
import math

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _compare(orc, sng, torch, x, p, want_screen=4):
    n = x.shape[0]
    m = p.draws(n)
    xg = torch.from_numpy(x).cuda()
    g = sng.build_graph(xg, p)
    st = g["stats"]
    assert st["map_screen"] == want_screen
    rp, col, band_pairs, _ = orc.build_rows(x, p.eps, p.seed, m,
                                            sample_all=p.sample_mode == 1, band_rel=BAND_F32)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    deg = orc.degrees(n, rp, col, mode=p.degree_mode)
    np.testing.assert_array_equal(g["deg"].cpu().numpy(), deg)
    assert st["band_pairs"] == band_pairs
    labels, core, cst = sng.cluster(xg, p, want_core=True)
    r = orc.cluster(x, p.eps, p.seed, m, p.min_pts, deg_mode=p.degree_mode,
                    sample_all=p.sample_mode == 1, band_rel=BAND_F32)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    for k in ("kept_edges", "band_pairs", "band_points", "cores", "clusters", "noise"):
        assert cst[k] == r[k], (k, cst[k], r[k])
    return st


def _params(sng, x, m, seed, **kw):
    d = x.shape[1]
    eps = float(np.float32(0.12 * math.sqrt(d)))
    return sng.Params(eps=eps, min_pts=4, m=m, seed=seed, flags=sng.SNG_FLAG_SCREEN8, **kw)


@pytest.mark.parametrize("n,d,m,budget", [(6000, 64, 90, 0), (6000, 64, 90, 2),
                                          (6000, 64, 90, 3), (4001, 64, 33, 0),
                                          (3000, 60, 7, 0), (4000, 32, 64, 0),
                                          (5000, 16, 90, 0), (3000, 3, 90, 0),
                                          (2500, 100, 90, 0), (2500, 100, 90, 2),
                                          (2000, 128, 90, 0), (1500, 64, 1, 0)])
def test_screen8_matches_oracle(orc, n, d, m, budget):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=7 * n + d)
    p = _params(sng, x, m, d + m, map_unroll=budget)
    st = _compare(orc, sng, torch, x, p)
    assert st["kept_edges"] > 0
    assert st["map_nch"] == (2 if d <= 64 else 4)


def test_screen8_wider_rows_use_the_bf16_copy(orc):
    """Past 128 values per row the flag falls back to the BF16 copy's
    tensor-core form (d <= 128 there too) or its CUDA-core form."""
    torch, sng = need_gpu()
    x = datagen.random_points(1500, 200, seed=3)
    p = _params(sng, x, 40, 3)
    _compare(orc, sng, torch, x, p, want_screen=1)


@pytest.mark.parametrize("deg_mode", [1, 2])
def test_screen8_degree_modes(orc, deg_mode):
    torch, sng = need_gpu()
    x = datagen.random_points(3001, 64, seed=deg_mode + 10)
    p = _params(sng, x, 70, 4, degree_mode=deg_mode)
    _compare(orc, sng, torch, x, p)


def test_screen8_all_pairs(orc):
    torch, sng = need_gpu()
    x = datagen.random_points(301, 48, seed=13)
    eps = float(np.float32(0.12 * math.sqrt(48)))
    p = sng.Params(eps=eps, min_pts=5, sample_mode=1, seed=1, flags=sng.SNG_FLAG_SCREEN8)
    _compare(orc, sng, torch, x, p)


def test_screen8_row_ranges_recompose(orc):
    torch, sng = need_gpu()
    n, d, m = 5000, 64, 80
    x = datagen.random_points(n, d, seed=21)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    whole = sng.build_graph(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2))
    wrp, wcol = whole["row_ptr"].cpu().numpy(), whole["col"].cpu().numpy()
    deg = np.zeros(n, dtype=np.int64)
    for lo, hi in ((0, 1999), (1999, 3001), (3001, 5000)):
        part = sng.build_graph(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2, row_begin=lo,
                                              row_end=hi, flags=sng.SNG_FLAG_SCREEN8))
        assert part["stats"]["map_screen"] == 4
        rp, col = part["row_ptr"].cpu().numpy(), part["col"].cpu().numpy()
        for i in (lo, lo + 1, (lo + hi) // 2, hi - 1):
            np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], wcol[wrp[i]:wrp[i + 1]])
        deg += part["deg"].cpu().numpy()
    np.testing.assert_array_equal(deg, whole["deg"].cpu().numpy())


def test_screen8_far_from_origin(orc):
    """Large norms against a small eps: the screen certifies little and most
    pairs are summed again in FP32."""
    torch, sng = need_gpu()
    n, d, m = 4000, 32, 60
    x = (datagen.random_points(n, d, seed=3) + 3000.0).astype(np.float32)
    p = _params(sng, x, m, 5)
    st = _compare(orc, sng, torch, x, p)
    assert st["screen_pairs"] > 0.5 * n * m


@pytest.mark.parametrize("scale_exp", [0, -40, 40, -45, 50])
def test_screen8_integer_ties_and_scales(orc, scale_exp):
    """Integer coordinates with eps^2 an integer put many pairs exactly on the
    ball's boundary; scaled by 2^-45 .. 2^50 they move the copy's scale
    exponent across its range."""
    torch, sng = need_gpu()
    n, d, m = 3000, 8, 200
    x = datagen.random_points(n, d, seed=7, kind="grid")
    s = np.float32(2.0 ** scale_exp)
    xs = (x * s).astype(np.float32)
    eps = float(np.float32(2.0 * s))
    p = sng.Params(eps=eps, min_pts=3, m=m, seed=9, flags=sng.SNG_FLAG_SCREEN8)
    st = _compare(orc, sng, torch, xs, p)
    assert st["band_pairs"] > 0


def test_screen8_scale_exponent_clamp(orc):
    """Values below 2^-54 ask for a scale exponent above 60, the clamp: the
    copy loses resolution, its per-row error bounds say so, and the result
    (here every pair within eps = 2^-49) is still the oracle's."""
    torch, sng = need_gpu()
    n, d, m = 2000, 8, 40
    x = (datagen.random_points(n, d, seed=4, kind="uniform") * np.float32(2.0 ** -54))
    x = x.astype(np.float32)
    p = sng.Params(eps=float(np.float32(2.0 ** -49)), min_pts=3, m=m, seed=1,
                   flags=sng.SNG_FLAG_SCREEN8)
    st = _compare(orc, sng, torch, x, p)
    assert st["kept_edges"] == n * m


def test_screen8_non_finite_rows(orc):
    torch, sng = need_gpu()
    n, d, m = 2000, 16, 50
    x = datagen.random_points(n, d, seed=11)
    x[5, 3] = np.inf
    x[17, 0] = np.nan
    x[400, 15] = -np.inf
    p = _params(sng, x, m, 2)
    _compare(orc, sng, torch, x, p)


def test_screen8_outlier_sets_the_scale(orc):
    """One coordinate 2^20 times larger than the rest fixes the copy's scale,
    so every other value lands near or below E4M3's subnormal range: the
    bound's absolute part keeps the decisions exact."""
    torch, sng = need_gpu()
    n, d, m = 3000, 32, 80
    x = datagen.random_points(n, d, seed=12)
    x[123, 7] = np.float32(2.0 ** 20)
    p = _params(sng, x, m, 6)
    _compare(orc, sng, torch, x, p)


def test_screen8_equals_plain_fp32_path(orc):
    """200,000 points of the headline mixture, 500 draws each (10^8 pairs):
    the FP8-screened gather gives the plain FP32 gather's CSR and degrees,
    and leaves a few percent of the pairs open."""
    torch, sng = need_gpu()
    n, d = 200_000, 64
    x = datagen.gaussian_mixture(n, d, 100, 0.02, seed=1)
    eps = datagen.eps_quantile(x, 0.01, 1_000_000, seed=1)
    xg = torch.from_numpy(x).cuda()
    base = dict(eps=eps, min_pts=10, m=500, seed=3)
    plain = sng.build_graph(xg, sng.Params(**base))
    scr = sng.build_graph(xg, sng.Params(**base, flags=sng.SNG_FLAG_SCREEN8))
    for k in ("row_ptr", "col", "deg", "core"):
        np.testing.assert_array_equal(scr[k].cpu().numpy(), plain[k].cpu().numpy(), err_msg=k)
    st = scr["stats"]
    assert st["map_screen"] == 4 and 0 < st["screen_pairs"] < 0.06 * n * 500
    rows = np.sort(np.random.default_rng(0).choice(n, 300, replace=False))
    rp, col, _, _ = orc.build_rows(x, eps, 3, 500, band_rel=BAND_F32, rows=rows)
    srp, scol = scr["row_ptr"].cpu().numpy(), scr["col"].cpu().numpy()
    for k, i in enumerate(rows):
        np.testing.assert_array_equal(scol[srp[i]:srp[i + 1]], col[rp[k]:rp[k + 1]])
