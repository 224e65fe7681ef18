"""The certified BF16 screen of FP32 points (SNG_FLAG_SCREEN16) against the
FP64 oracle: the screen decides a pair from a BF16 copy of the points only
where the copy's rounding cannot change the decision, so the graph (row
pointers, columns, degrees, band counts) and the labels must be exactly the
oracle's -- for the direct and the tiled gather, every compiled BF16 mapping
shape, rows that force every pair open (far from the origin, non-finite,
tiny or huge values), exact ties at eps, and the headline workload at full
size."""
import math

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _graph(sng, xg, p):
    g = sng.build_graph(xg, p)
    return {k: g[k].cpu().numpy() for k in ("row_ptr", "col", "deg", "core")}, g["stats"]


def _check_exact(orc, sng, torch, x, p, m, min_pts, tiled_k=0, mma=False):
    xg = torch.from_numpy(x).cuda()
    flags = sng.SNG_FLAG_SCREEN16 | (sng.SNG_FLAG_TILED if tiled_k else 0)
    if mma:
        flags |= sng.SNG_FLAG_SCREEN_MMA
    if mma == "tc05":
        flags |= sng.SNG_FLAG_TCGEN05
    q = sng.Params(**{**p.__dict__, "flags": flags, "map_tile": tiled_k})
    g, st = _graph(sng, xg, q)
    d = x.shape[1]
    want = (3 if mma == "tc05" and d <= 64 else 2) if mma and d <= 128 else 1
    assert st["map_screen"] == want
    rp, col, bpairs, _ = orc.build_rows(x, p.eps, p.seed, m, band_rel=BAND_F32)
    np.testing.assert_array_equal(g["row_ptr"], rp)
    np.testing.assert_array_equal(g["col"], col)
    assert st["band_pairs"] == bpairs
    labels, core, cst = sng.cluster(xg, q, want_core=True)
    r = orc.cluster(x, p.eps, p.seed, m, min_pts, band_rel=BAND_F32)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    assert cst["band_points"] == r["band_points"]
    return st


@pytest.mark.parametrize("tiled_k", [0, 3])
@pytest.mark.parametrize("n,d,group,unroll", [(6000, 64, 0, 0), (6000, 64, 8, 2),
                                              (5000, 64, 8, 4), (4000, 128, 0, 0),
                                              (4000, 32, 0, 0), (3000, 60, 0, 0),
                                              (5000, 16, 0, 0), (3000, 3, 0, 0),
                                              (2500, 100, 16, 2)])
def test_screen_matches_oracle(orc, n, d, group, unroll, tiled_k):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    m = 90
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=d, map_group=group, map_unroll=unroll)
    st = _check_exact(orc, sng, torch, x, p, m, 4, tiled_k)
    assert st["kept_edges"] > 0
    # the tiled form runs where a tile mapping is compiled for the BF16 copy
    # (full rows of 64 or 128 values); elsewhere the direct gather does
    if tiled_k and d in (64, 128):
        assert st["map_tiles"] == tiled_k


@pytest.mark.parametrize("n,d,budget", [(6000, 64, 0), (6000, 64, 2), (6000, 64, 4),
                                        (4000, 128, 0), (4000, 128, 3), (4000, 32, 0),
                                        (4000, 32, 4), (3000, 60, 0), (5000, 16, 0),
                                        (3000, 3, 0), (2500, 100, 0), (2000, 200, 0)])
def test_screen_tensor_cores_match_oracle(orc, n, d, budget):
    """The tensor-core form (SNG_FLAG_SCREEN_MMA): 2, 4 or 8 k-tiles of 16
    values per row (d <= 32, 64, 128; beyond that the CUDA-core screen), with
    registers budgeted for 2, 3 or 4 resident blocks per SM (map_unroll)."""
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=3 * n + d)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    m = 90
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=d + 1, map_unroll=budget)
    st = _check_exact(orc, sng, torch, x, p, m, 4, mma=True)
    assert st["kept_edges"] > 0


@pytest.mark.parametrize("mma", [False, True, "tc05"])
def test_screen_open_pairs_far_from_origin(orc, mma):
    """Points offset far from the origin make every norm bound large, so the
    screen certifies little and most pairs are summed again in FP32: the
    result is still the oracle's."""
    torch, sng = need_gpu()
    n, d, m = 4000, 32, 60
    x = (datagen.random_points(n, d, seed=3) + 3000.0).astype(np.float32)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=5)
    st = _check_exact(orc, sng, torch, x, p, m, 4, mma=mma)
    assert st["screen_pairs"] > 0.5 * n * m


@pytest.mark.parametrize("mma", [False, True, "tc05"])
def test_screen_integer_ties_and_mixed_scales(orc, mma):
    """Integer coordinates (exact in every format) with eps^2 an integer put
    many pairs exactly on the ball's boundary (kept: closed ball), all of
    them in the reported band; the same points scaled by 2^-40 and 2^40 test
    tiny and large norms."""
    torch, sng = need_gpu()
    n, d, m = 3000, 8, 200
    x = datagen.random_points(n, d, seed=7, kind="grid")
    eps = 2.0                                    # eps^2 = 4 = a sum of integer squares
    p = sng.Params(eps=eps, min_pts=3, m=m, seed=9)
    st = _check_exact(orc, sng, torch, x, p, m, 3, mma=mma)
    assert st["band_pairs"] > 0
    for scale in (2.0 ** -40, 2.0 ** 40):
        xs = (x * np.float32(scale)).astype(np.float32)
        ps = sng.Params(eps=float(np.float32(eps * scale)), min_pts=3, m=m, seed=9)
        _check_exact(orc, sng, torch, xs, ps, m, 3, mma=mma)


@pytest.mark.parametrize("mma", [False, True, "tc05"])
def test_screen_non_finite_rows(orc, mma):
    """Rows holding inf or NaN give unbounded norms, which certify nothing:
    their pairs (and, through the maximum norm, every pair) are decided from
    the FP32 points, as the oracle decides them (a NaN or infinite distance
    is never within eps)."""
    torch, sng = need_gpu()
    n, d, m = 2000, 16, 50
    x = datagen.random_points(n, d, seed=11)
    x[5, 3] = np.inf
    x[17, 0] = np.nan
    x[400, 15] = -np.inf
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=2)
    _check_exact(orc, sng, torch, x, p, m, 4, mma=mma)


@pytest.mark.parametrize("tiled_k,mma", [(0, False), (3, False), (0, True), (0, "tc05")])
def test_screen_equals_plain_fp32_path(orc, tiled_k, mma):
    """On a Gaussian mixture shaped like the headline workload (smaller n)
    the screened and the plain FP32 gathers give the same CSR, degrees and
    labels."""
    torch, sng = need_gpu()
    n, d = 200_000, 64
    x = datagen.gaussian_mixture(n, d, 100, 0.02, seed=1)
    eps = datagen.eps_quantile(x, 0.01, 1_000_000, seed=1)
    xg = torch.from_numpy(x).cuda()
    base = dict(eps=eps, min_pts=10, m=500, seed=3)
    plain, _ = _graph(sng, xg, sng.Params(**base))
    flags = sng.SNG_FLAG_SCREEN16 | (sng.SNG_FLAG_TILED if tiled_k else 0)
    flags |= sng.SNG_FLAG_SCREEN_MMA if mma else 0
    flags |= sng.SNG_FLAG_TCGEN05 if mma == "tc05" else 0
    scr, st = _graph(sng, xg, sng.Params(**base, flags=flags, map_tile=tiled_k))
    for k in plain:
        np.testing.assert_array_equal(scr[k], plain[k], err_msg=k)
    want = 3 if mma == "tc05" else 2 if mma else 1
    assert st["map_screen"] == want and 0 < st["screen_pairs"] < 0.02 * n * 500
    rows = np.sort(np.random.default_rng(0).choice(n, 300, replace=False))
    rp, col, _, _ = orc.build_rows(x, eps, 3, 500, band_rel=BAND_F32, rows=rows)
    for k, i in enumerate(rows):
        np.testing.assert_array_equal(scr["col"][scr["row_ptr"][i]:scr["row_ptr"][i + 1]],
                                      col[rp[k]:rp[k + 1]])


def test_screen_bf16_points_ignore_the_flag(orc):
    """The flag concerns FP32 points; BF16 points run their own form."""
    torch, sng = need_gpu()
    n, d = 3000, 32
    x = datagen.random_points(n, d, seed=4)
    bits = datagen.bf16_round(x)
    xo = datagen.bf16_to_f32(bits)
    xb = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    master = torch.from_numpy(xo).cuda()
    eps = float(np.float32(0.12 * math.sqrt(d)))
    lab, st = sng.cluster(xb, sng.Params(eps=eps, min_pts=4, m=40, seed=1,
                                         flags=sng.SNG_FLAG_SCREEN16), x_master=master)
    ref, _ = sng.cluster(xb, sng.Params(eps=eps, min_pts=4, m=40, seed=1), x_master=master)
    assert st["map_screen"] == 0
    assert torch.equal(lab, ref)
