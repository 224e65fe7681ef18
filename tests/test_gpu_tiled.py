"""The L2-tiled form of step 2 (SNG_FLAG_TILED) against the oracle and the
direct gather: CSR, degrees, band counts and labels equal, for several slice
counts, full-row and general mappings, FP32 and BF16, the three degree
definitions, every pair queried, and source-row ranges."""
import math

import numpy as np
import pytest

from gpu_util import BAND_BF16, BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _graph(sng, xg, p, master=None):
    g = sng.build_graph(xg, p, x_master=master)
    return {k: g[k].cpu().numpy() for k in ("row_ptr", "col", "deg", "core")}, g["stats"]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("n,d,tiles", [(5000, 64, 0), (7000, 64, 3), (4000, 128, 2),
                                       (6000, 32, 8), (3000, 60, 4), (5000, 16, 5),
                                       (6000, 64, 17), (9000, 64, 32), (4000, 128, 40)])
def test_tiled_graph_matches_oracle_and_direct(orc, dtype, n, d, tiles):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d + tiles)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    m = 90
    if dtype == "bf16":
        bits = datagen.bf16_round(x)
        xo = datagen.bf16_to_f32(bits)
        xg = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
        master, band = torch.from_numpy(xo).cuda(), BAND_BF16
    else:
        xo, xg, master, band = x, torch.from_numpy(x).cuda(), None, BAND_F32
    base = dict(eps=eps, min_pts=4, m=m, seed=d)
    tiled, st = _graph(sng, xg, sng.Params(**base, flags=sng.SNG_FLAG_TILED, map_tile=tiles),
                       master)
    direct, _ = _graph(sng, xg, sng.Params(**base), master)
    for k in tiled:
        np.testing.assert_array_equal(tiled[k], direct[k], err_msg=k)
    rp, col, bpairs, _ = orc.build_rows(xo, eps, d, m, band_rel=band)
    np.testing.assert_array_equal(tiled["row_ptr"], rp)
    np.testing.assert_array_equal(tiled["col"], col)
    assert st["band_pairs"] == bpairs
    labels, _ = sng.cluster(xg, sng.Params(**base, flags=sng.SNG_FLAG_TILED, map_tile=tiles),
                            x_master=master)
    r = orc.cluster(xo, eps, d, m, 4, band_rel=band)
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])


@pytest.mark.parametrize("deg_mode", [0, 1, 2])
def test_tiled_degree_modes_and_every_pair(orc, deg_mode):
    torch, sng = need_gpu()
    n, d = 2500, 32
    x = datagen.random_points(n, d, seed=deg_mode)
    eps = float(np.float32(0.1 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    for extra in (dict(m=150, seed=3), dict(sample_mode=1)):
        p = sng.Params(eps=eps, min_pts=4, degree_mode=deg_mode, flags=sng.SNG_FLAG_TILED,
                       map_tile=3, **extra)
        labels, core, st = sng.cluster(xg, p, want_core=True)
        m = n - 1 if extra.get("sample_mode") else 150
        r = orc.cluster(x, eps, extra.get("seed", 0), m, 4, deg_mode=deg_mode,
                        sample_all=bool(extra.get("sample_mode")), band_rel=BAND_F32)
        np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
        np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
        assert st["kept_edges"] == r["kept_edges"]


def test_tiled_row_ranges_recompose(orc):
    """Source-row shards built in the tiled form give the rows of the whole
    graph and sum to its degrees (the multi-GPU exchange's inputs)."""
    torch, sng = need_gpu()
    n, d, m = 6000, 64, 80
    x = datagen.random_points(n, d, seed=9)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    whole, _ = _graph(sng, xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2))
    deg = np.zeros(n, dtype=np.int64)
    for lo, hi in ((0, 2500), (2500, 6000)):
        part, _ = _graph(sng, xg, sng.Params(eps=eps, min_pts=4, m=m, seed=2, row_begin=lo,
                                             row_end=hi, flags=sng.SNG_FLAG_TILED, map_tile=4))
        rp = part["row_ptr"]
        for i in (lo, (lo + hi) // 2, hi - 1):
            np.testing.assert_array_equal(part["col"][rp[i]:rp[i + 1]],
                                          whole["col"][whole["row_ptr"][i]:whole["row_ptr"][i + 1]])
        deg += part["deg"]
    np.testing.assert_array_equal(deg, whole["deg"])


@pytest.mark.parametrize("m", [1023, 1024, 1025, 2600])
def test_tiled_rows_past_the_partition_cache(orc, m):
    """Rows of up to 1024 draws keep their partners in shared memory between
    the partition's passes; longer rows hash again.  Both sides of the limit
    give the direct gather's graph and the oracle's rows."""
    torch, sng = need_gpu()
    n, d = 3000, 64
    x = datagen.random_points(n, d, seed=m)
    eps = float(np.float32(0.1 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    base = dict(eps=eps, min_pts=4, m=m, seed=7)
    tiled, st = _graph(sng, xg, sng.Params(**base, flags=sng.SNG_FLAG_TILED, map_tile=5))
    direct, _ = _graph(sng, xg, sng.Params(**base))
    for k in tiled:
        np.testing.assert_array_equal(tiled[k], direct[k], err_msg=k)
    rp, col, bpairs, _ = orc.build_rows(x, eps, 7, m, band_rel=BAND_F32)
    np.testing.assert_array_equal(tiled["row_ptr"], rp)
    np.testing.assert_array_equal(tiled["col"], col)
    assert st["band_pairs"] == bpairs and st["kept_edges"] > 0


@pytest.mark.parametrize("group,unroll", [(2, 1), (2, 2), (4, 4), (8, 2), (4, 2)])
def test_tiled_lane_groups_and_steps(orc, group, unroll):
    """FP32 rows of 64 values tested by 2, 4 or 8 lanes per pair with 1, 2 or
    4 partner steps in flight: the group reduction hands each lane whole
    sums of different steps (fewer or more steps than lanes), and every
    arrangement gives the default mapping's graph and the oracle's rows."""
    torch, sng = need_gpu()
    n, d, m = 6000, 64, 140
    x = datagen.random_points(n, d, seed=20 + unroll + group)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    base = dict(eps=eps, min_pts=4, m=m, seed=11)
    tiled, st = _graph(sng, xg, sng.Params(**base, flags=sng.SNG_FLAG_TILED, map_tile=3,
                                           map_group=group, map_unroll=unroll))
    assert st["map_group"] == group
    direct, _ = _graph(sng, xg, sng.Params(**base))
    for k in tiled:
        np.testing.assert_array_equal(tiled[k], direct[k], err_msg=k)
    rp, col, bpairs, _ = orc.build_rows(x, eps, 11, m, band_rel=BAND_F32)
    np.testing.assert_array_equal(tiled["col"], col)
    assert st["band_pairs"] == bpairs


def test_tiled_reports_its_slices_and_falls_back(orc):
    """stats map_tiles is the slice count when the tiled form ran and 0 where
    it does not apply (cosine similarity; the no-sync form, which must stay
    capturable in a CUDA graph) -- those calls run the direct gather and give
    the same labels."""
    torch, sng = need_gpu()
    n, d, m = 4000, 64, 100
    x = datagen.random_points(n, d, seed=31)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=5, flags=sng.SNG_FLAG_TILED, map_tile=3)
    labels, st = sng.cluster(xg, p)
    assert st["map_tiles"] == 3
    _, st_direct = sng.cluster(xg, sng.Params(eps=eps, min_pts=4, m=m, seed=5))
    assert st_direct["map_tiles"] == 0
    _, st_cos = sng.cluster(xg, sng.Params(eps=0.2, min_pts=4, m=m, seed=5, metric=2,
                                           flags=sng.SNG_FLAG_TILED, map_tile=3))
    assert st_cos["map_tiles"] == 0
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        sng.cluster_async(xg, p, out)                   # warm-up off the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sng.cluster_async(xg, p, out)
    out.fill_(-7)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, labels)
    r = orc.cluster(x, eps, 5, m, 4, band_rel=BAND_F32)
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])


@pytest.mark.parametrize("ld", [64, 68, 96])
def test_tiled_texture_chunk_on_padded_rows(orc, ld):
    """FP32 rows of 64 values take one 16-byte chunk per partner through the
    texture unit.  Rows with a padded stride, in a buffer that ends right
    after the last row's 64 values (padding holding NaN), give the oracle's
    graph."""
    torch, sng = need_gpu()
    n, d, m = 5000, 64, 120
    x = datagen.random_points(n, d, seed=ld)
    flat = torch.full(((n - 1) * ld + d,), float("nan"), dtype=torch.float32, device="cuda")
    xg = flat.as_strided((n, d), (ld, 1))
    xg.copy_(torch.from_numpy(x))
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=3, flags=sng.SNG_FLAG_TILED, map_tile=4)
    g, st = _graph(sng, xg, p)
    assert st["map_tiles"] == 4 and st["map_group"] == 4 and st["map_unroll"] == 2
    rp, col, bpairs, _ = orc.build_rows(x, eps, 3, m, band_rel=BAND_F32)
    np.testing.assert_array_equal(g["row_ptr"], rp)
    np.testing.assert_array_equal(g["col"], col)
    assert st["band_pairs"] == bpairs


@pytest.mark.parametrize("pinned", [False, True])
def test_tiled_host_buffer_call_overlaps_copy(pinned):
    """sng_cluster_host in the tiled form: the partition reads no
    coordinates, so it runs while the points are still being copied in (four
    pieces on side streams); the tile tests wait for the copies.  Labels,
    core flags and counts equal the device call's."""
    torch, sng = need_gpu()
    n, d, m = 400_000, 64, 60
    x = datagen.gaussian_mixture(n, d, 40, 0.02, seed=8)
    p = sng.Params(eps=8.0, min_pts=6, m=m, seed=6, flags=sng.SNG_FLAG_TILED)
    ref, ref_core, st_ref = sng.cluster(torch.from_numpy(x).cuda(), p, want_core=True)
    assert st_ref["map_tiles"] >= 2
    xt = torch.from_numpy(x)
    if pinned:
        xt = xt.pin_memory()
    for _ in range(2):
        labels, core, st = sng.cluster_host(xt, p, want_core=True)
        np.testing.assert_array_equal(labels, ref.cpu().numpy())
        np.testing.assert_array_equal(core, ref_core.cpu().numpy())
        assert st["map_tiles"] == st_ref["map_tiles"]
        assert st["kept_edges"] == st_ref["kept_edges"] and st["kept_edges"] > 0


def test_tiled_falls_back_when_its_buckets_cannot_be_allocated(orc):
    """A failed allocation of the tiled form's buckets, runs or counters
    (host-side injection: the k-th scratch allocation of the call fails; the
    seven before them are the graph's own) makes the call run the direct
    gather: same labels, map_tiles 0, no error."""
    import os
    torch, sng = need_gpu()
    n, d, m = 4000, 64, 80
    x = datagen.random_points(n, d, seed=44)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    p = sng.Params(eps=eps, min_pts=4, m=m, seed=9, flags=sng.SNG_FLAG_TILED, map_tile=3)
    ref, st_ref = sng.cluster(xg, p)
    assert st_ref["map_tiles"] == 3
    for k in (8, 9, 14):
        os.environ["SNG_FAULT_ALLOC"] = str(k)
        try:
            got, st = sng.cluster(xg, p)
        finally:
            del os.environ["SNG_FAULT_ALLOC"]
        assert st["map_tiles"] == 0, k
        assert torch.equal(got, ref), k
    r = orc.cluster(x, eps, 9, m, 4, band_rel=BAND_F32)
    np.testing.assert_array_equal(ref.cpu().numpy(), r["labels"])
    _, st_again = sng.cluster(xg, p)
    assert st_again["map_tiles"] == 3
