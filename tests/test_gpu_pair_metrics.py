"""Step 2 with the Manhattan (L1) and Chebyshev (L-inf) distances against the
FP64 oracle: CSR, degrees, band counts and labels bit-exact, over the FP32
points and through the BF16 screen (SNG_FLAG_SCREEN16: pairs decided on the
copy where its error bounds allow, the rest queued and decided from the FP32
points) -- over row widths that take the 16-byte group layout (source row in
registers up to 64 values, reloaded past it) and the scalar loads, padded
rows holding junk, integer coordinates with many pairs exactly at eps (kept,
counted in the band; through the screen more open pairs than its queue
holds), rows with NaN and inf, every degree mode, every-pair sampling and
source-row ranges, and the screen at 10^6 points on sampled rows; and the
forms these metrics do not take (BF16 points, the tiled gather, the
tensor-core screens) rejected or ignored."""
import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu

L1, LINF = 3, 4
SCREEN16 = 32


def _flags(screen):
    return SCREEN16 if screen else 0


def _eps(x, metric, q, seed=0):
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    i, j = rng.integers(0, n, 20000), rng.integers(0, n, 20000)
    diff = np.abs(x[i].astype(np.float64) - x[j].astype(np.float64))
    v = diff.sum(axis=1) if metric == L1 else diff.max(axis=1)
    return float(np.float32(np.quantile(v, q)))


def _compare(orc, sng, torch, x, xg, p):
    n = x.shape[0]
    m = p.draws(n)
    g = sng.build_graph(xg, p)
    rp, col, band_pairs, _ = orc.build_rows(x, p.eps, p.seed, m, sample_all=p.sample_mode == 1,
                                            band_rel=BAND_F32, metric=p.metric)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    np.testing.assert_array_equal(g["deg"].cpu().numpy(),
                                  orc.degrees(n, rp, col, mode=p.degree_mode))
    assert g["stats"]["band_pairs"] == band_pairs
    labels, core, st = sng.cluster(xg, p, want_core=True)
    r = orc.cluster(x, p.eps, p.seed, m, p.min_pts, deg_mode=p.degree_mode,
                    sample_all=p.sample_mode == 1, band_rel=BAND_F32, metric=p.metric)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    for k in ("kept_edges", "band_pairs", "band_points", "cores", "clusters", "noise"):
        assert st[k] == r[k], (k, st[k], r[k])
    return st


@pytest.mark.parametrize("screen", [False, True])
@pytest.mark.parametrize("metric", [L1, LINF])
@pytest.mark.parametrize("n,d", [(400, 1), (700, 3), (1000, 4), (900, 7), (1200, 16),
                                 (900, 24), (800, 32), (2000, 64), (800, 65), (600, 128),
                                 (500, 130), (400, 200)])
def test_pair_metric_graph_and_labels_match_oracle(orc, metric, n, d, screen):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d + metric)
    p = sng.Params(eps=_eps(x, metric, 0.03, seed=d), min_pts=3, m=min(150, 3 * n), seed=d,
                   metric=metric, flags=_flags(screen))
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["kept_edges"] > 0
    assert st["map_screen"] == (1 if screen else 0)
    if screen:
        # the copy decides most pairs
        assert st["screen_pairs"] < 0.2 * n * p.draws(n)


@pytest.mark.parametrize("screen", [False, True])
@pytest.mark.parametrize("metric", [L1, LINF])
@pytest.mark.parametrize("d,ld,fill", [(3, 4, float("nan")), (8, 12, float("inf")),
                                       (64, 72, -1e30)])
def test_pair_metric_padded_rows_ignore_padding(orc, metric, d, ld, fill, screen):
    torch, sng = need_gpu()
    n = 800
    x = datagen.random_points(n, d, seed=ld)
    buf = torch.full((n, ld), fill, dtype=torch.float32, device="cuda")
    buf[:, :d] = torch.from_numpy(x).cuda()
    p = sng.Params(eps=_eps(x, metric, 0.05), min_pts=3, m=100, seed=5, metric=metric,
                   flags=_flags(screen))
    _compare(orc, sng, torch, x, buf[:, :d], p)


@pytest.mark.parametrize("screen", [False, True])
@pytest.mark.parametrize("metric", [L1, LINF])
def test_pair_metric_integer_ties_kept_and_counted(orc, metric, screen):
    torch, sng = need_gpu()
    rng = np.random.default_rng(3)
    n, d = 2500, 4
    x = rng.integers(0, 5, (n, d)).astype(np.float32)
    eps = 3.0 if metric == L1 else 1.0
    p = sng.Params(eps=eps, min_pts=4, m=200, seed=2, metric=metric, flags=_flags(screen))
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["band_pairs"] > 1000
    if screen:
        # every tie is open: more than the queue's n m / 32 entries, so the
        # gather decides the rest itself
        assert st["screen_pairs"] > n * 200 // 32


@pytest.mark.parametrize("screen", [False, True])
@pytest.mark.parametrize("metric", [L1, LINF])
def test_pair_metric_nonfinite_rows(orc, metric, screen):
    torch, sng = need_gpu()
    n, d = 1500, 8
    x = datagen.random_points(n, d, seed=9)
    x[3, 2] = np.nan
    x[11, 0] = np.inf
    x[13, 5] = -np.inf
    x[17] = np.inf                      # inf - inf = NaN against row 11's inf
    x[19, 1] = 3.4e38                   # rounds to inf in BF16
    p = sng.Params(eps=_eps(x[20:], metric, 0.05), min_pts=3, m=200, seed=2, metric=metric,
                   flags=_flags(screen))
    _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)


@pytest.mark.parametrize("screen", [False, True])
@pytest.mark.parametrize("metric", [L1, LINF])
@pytest.mark.parametrize("deg_mode", [0, 1, 2])
def test_pair_metric_degree_modes_and_sample_all(orc, metric, deg_mode, screen):
    torch, sng = need_gpu()
    n, d = 500, 6
    x = datagen.random_points(n, d, seed=4)
    eps = _eps(x, metric, 0.05)
    f = _flags(screen)
    for p in (sng.Params(eps=eps, min_pts=4, m=300, seed=3, metric=metric, degree_mode=deg_mode,
                         flags=f),
              sng.Params(eps=eps, min_pts=4, sample_mode=1, metric=metric,
                         degree_mode=deg_mode, flags=f)):
        _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)


@pytest.mark.parametrize("screen", [False, True])
@pytest.mark.parametrize("metric", [L1, LINF])
def test_pair_metric_row_ranges_recompose(orc, metric, screen):
    torch, sng = need_gpu()
    n, d, m = 3000, 16, 80
    x = datagen.random_points(n, d, seed=21)
    eps = _eps(x, metric, 0.05)
    xg = torch.from_numpy(x).cuda()
    f = _flags(screen)
    whole = sng.build_graph(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2, metric=metric,
                                           flags=f))
    wrp, wcol = whole["row_ptr"].cpu().numpy(), whole["col"].cpu().numpy()
    deg = np.zeros(n, dtype=np.int64)
    for lo, hi in ((0, 1201), (1201, 3000)):
        part = sng.build_graph(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2, metric=metric,
                                              row_begin=lo, row_end=hi, flags=f))
        rp, col = part["row_ptr"].cpu().numpy(), part["col"].cpu().numpy()
        for i in (lo, (lo + hi) // 2, hi - 1):
            np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], wcol[wrp[i]:wrp[i + 1]])
        deg += part["deg"].cpu().numpy()
    np.testing.assert_array_equal(deg, whole["deg"].cpu().numpy())


def test_pair_metric_rejections_and_ignored_flags(orc):
    torch, sng = need_gpu()
    n, d = 600, 8
    x = datagen.random_points(n, d, seed=1)
    xf = torch.from_numpy(x).cuda()
    with pytest.raises(sng.SngError) as e:          # BF16 points
        sng.cluster(xf.to(torch.bfloat16), sng.Params(eps=0.5, min_pts=3, m=50, metric=L1),
                    x_master=xf)
    assert e.value.status == sng.SNG_EINVAL
    with pytest.raises(sng.SngError) as e:          # eps below the radius range
        sng.cluster(xf, sng.Params(eps=1e-20, min_pts=3, m=50, metric=LINF))
    assert e.value.status == sng.SNG_EINVAL
    # the tiled form and the tensor-core screens do not apply: the BF16
    # screen on CUDA cores runs for either screen flag
    for f in (sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA | sng.SNG_FLAG_TILED,
              sng.SNG_FLAG_SCREEN8 | sng.SNG_FLAG_TCGEN05):
        p = sng.Params(eps=_eps(x, L1, 0.05), min_pts=3, m=60, seed=1, metric=L1, flags=f)
        st = _compare(orc, sng, torch, x, xf, p)
        assert st["map_screen"] == 1 and st["map_tiles"] == 0
    p = sng.Params(eps=_eps(x, L1, 0.05), min_pts=3, m=60, seed=1, metric=L1,
                   flags=sng.SNG_FLAG_TILED)
    st = _compare(orc, sng, torch, x, xf, p)
    assert st["map_screen"] == 0 and st["map_tiles"] == 0


@pytest.mark.parametrize("metric", [L1, LINF])
def test_pair_metric_screen_at_a_million_points(orc, metric):
    """The screen at the headline's points (n = 10^6, d = 64 mixture, m =
    1000, eps at the 1% quantile of the metric): sampled rows bit-exact
    against the oracle, the whole CSR and the labels equal to the plain pair
    gather's, most pairs decided on the copy."""
    torch, sng = need_gpu()
    n, d, m = 1_000_000, 64, 1000
    x = datagen.gaussian_mixture(n, d, 100, 0.02, seed=0)
    eps = _eps(x, metric, 0.01)
    xg = torch.from_numpy(x).cuda()
    base = dict(eps=eps, min_pts=10, m=m, seed=0, metric=metric)
    g1 = sng.build_graph(xg, sng.Params(**base, flags=SCREEN16))
    assert g1["stats"]["map_screen"] == 1
    assert g1["stats"]["screen_pairs"] < 0.01 * n * m
    rp1, col1 = g1["row_ptr"].cpu().numpy(), g1["col"].cpu().numpy()
    rows = np.random.default_rng(7).choice(n, 1500, replace=False)
    rows.sort()
    rp, col, _, _ = orc.build_rows(x, eps, 0, m, band_rel=BAND_F32, rows=rows, metric=metric)
    for k, i in enumerate(rows):
        np.testing.assert_array_equal(col1[rp1[i]:rp1[i + 1]], col[rp[k]:rp[k + 1]])
    g0 = sng.build_graph(xg, sng.Params(**base))
    np.testing.assert_array_equal(g0["row_ptr"].cpu().numpy(), rp1)
    np.testing.assert_array_equal(g0["col"].cpu().numpy(), col1)
    np.testing.assert_array_equal(g0["deg"].cpu().numpy(), g1["deg"].cpu().numpy())
    assert g0["stats"]["band_pairs"] == g1["stats"]["band_pairs"]
    del g0, g1
    l1, _ = sng.cluster(xg, sng.Params(**base, flags=SCREEN16))
    l0, _ = sng.cluster(xg, sng.Params(**base))
    assert torch.equal(l0, l1)
