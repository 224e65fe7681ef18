"""The screened gather with TMA row gathers and tcgen05 dot products
(SNG_FLAG_TCGEN05) against the FP64 oracle.  The kernel works on four source
rows per CTA and 32 draws per row per stage, so the cases put ragged ends on
both: point counts that are not multiples of 4, draw counts below, at and
past multiples of 32, row ranges that start mid-group, every degree mode,
the all-pairs draw, and rows narrower than the 64 values the copy holds."""
import math

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _flags(sng):
    return sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA | sng.SNG_FLAG_TCGEN05


def _compare(orc, sng, torch, x, p):
    """CSR, degrees, core flags, labels and counters equal to the oracle's."""
    n = x.shape[0]
    m = p.draws(n)
    xg = torch.from_numpy(x).cuda()
    g = sng.build_graph(xg, p)
    st = g["stats"]
    assert st["map_screen"] == 3
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


@pytest.mark.parametrize("n,d,m", [(6000, 64, 90), (4001, 64, 90), (4002, 64, 32),
                                   (4003, 64, 33), (3000, 60, 7), (4000, 32, 64),
                                   (5000, 16, 90), (3000, 3, 90), (2003, 64, 300),
                                   (1500, 64, 1)])
def test_tcgen05_gather_matches_oracle(orc, n, d, m):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=5 * n + d)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=d + m, flags=_flags(sng))
    st = _compare(orc, sng, torch, x, p)
    assert st["kept_edges"] > 0 and st["map_group"] == 128


@pytest.mark.parametrize("deg_mode", [1, 2])
def test_tcgen05_degree_modes(orc, deg_mode):
    torch, sng = need_gpu()
    n, d, m = 3001, 64, 70
    x = datagen.random_points(n, d, seed=deg_mode)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=3, m=m, seed=4, degree_mode=deg_mode, flags=_flags(sng))
    _compare(orc, sng, torch, x, p)


def test_tcgen05_all_pairs(orc):
    """sample_mode 1: every row draws every other point (n - 1 draws)."""
    torch, sng = need_gpu()
    n, d = 301, 48
    x = datagen.random_points(n, d, seed=13)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=5, sample_mode=1, seed=1, flags=_flags(sng))
    _compare(orc, sng, torch, x, p)


def test_tcgen05_mixture_at_the_paper_rate(orc):
    """A Gaussian mixture at s = 0.01 (m = 400 of 40,000 points), the regime
    of the paper's experiments, where most kept pairs are certified."""
    torch, sng = need_gpu()
    n, d = 40_000, 64
    x = datagen.gaussian_mixture(n, d, 20, 0.02, seed=2)
    eps = datagen.eps_quantile(x, 0.01, 200_000, seed=2)
    p = sng.Params(eps=eps, min_pts=10, s=0.01, seed=7, flags=_flags(sng))
    st = _compare(orc, sng, torch, x, p)
    assert st["screen_pairs"] < 0.05 * n * p.draws(n)


def test_tcgen05_row_ranges_recompose(orc):
    """Source-row shards whose bounds are not multiples of four give the rows
    of the whole graph and sum to its degrees."""
    torch, sng = need_gpu()
    n, d, m = 5000, 64, 80
    x = datagen.random_points(n, d, seed=21)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    fl = _flags(sng)
    whole = sng.build_graph(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2))
    wrp, wcol = whole["row_ptr"].cpu().numpy(), whole["col"].cpu().numpy()
    deg = np.zeros(n, dtype=np.int64)
    for lo, hi in ((0, 1999), (1999, 3001), (3001, 5000)):
        part = sng.build_graph(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2, row_begin=lo,
                                              row_end=hi, flags=fl))
        assert part["stats"]["map_screen"] == 3
        rp, col = part["row_ptr"].cpu().numpy(), part["col"].cpu().numpy()
        for i in (lo, lo + 1, (lo + hi) // 2, hi - 1):
            np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], wcol[wrp[i]:wrp[i + 1]])
        deg += part["deg"].cpu().numpy()
    np.testing.assert_array_equal(deg, whole["deg"].cpu().numpy())


def test_tcgen05_wider_rows_use_the_mma_form(orc):
    """Past 64 values per row the flag leaves the mma.sync form in charge."""
    torch, sng = need_gpu()
    n, d, m = 2000, 96, 40
    x = datagen.random_points(n, d, seed=3)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=3, flags=_flags(sng))
    g = sng.build_graph(torch.from_numpy(x).cuda(), p)
    assert g["stats"]["map_screen"] == 2
    rp, col, _, _ = orc.build_rows(x, eps, 3, m, band_rel=BAND_F32)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
