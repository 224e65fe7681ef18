"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Integer outputs (partners, CSR, degrees, core mask,
labels) must be bit-exact; FP32 inputs give FP64 decisions on every pair
thanks to the in-kernel FP64 recheck inside the guard band."""
import math

import numpy as np
import pytest

from gpu_util import BAND_BF16, BAND_F32, need_gpu, padded
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [2, 3, 17, 1000, 123_457, 2**31 - 1])
def test_partners_match_oracle(orc, n):
    torch, sng = need_gpu()
    rows = min(n, 64)
    for seed in (0, 12345, 2**64 - 1):
        for i0 in (0, max(0, n - rows)):
            g = sng.sample_partners(n, seed, i0, rows, 97).cpu().numpy()
            o = orc.partners(seed, n, i0, rows, 97)
            np.testing.assert_array_equal(g, o)


def test_partners_sample_all(orc):
    torch, sng = need_gpu()
    g = sng.sample_partners(50, 0, 0, 50, 49, sample_all=True).cpu().numpy()
    np.testing.assert_array_equal(g, orc.partners(0, 50, 0, 50, 49, sample_all=True))


def _compare_graph(orc, x_np, xg, p, sng, master=None):
    n = x_np.shape[0]
    m = p.draws(n)
    g = sng.build_graph(xg, p, x_master=master)
    rp, col, band_pairs, bp = orc.build_rows(x_np, p.eps, p.seed, m,
                                             sample_all=p.sample_mode == 1, band_rel=BAND_F32)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    deg = orc.degrees(n, rp, col, mode=p.degree_mode)
    np.testing.assert_array_equal(g["deg"].cpu().numpy(), deg)
    np.testing.assert_array_equal(g["core"].cpu().numpy(), (deg >= p.min_pts).astype(np.uint8))
    assert g["stats"]["kept_edges"] == col.size
    assert g["stats"]["band_pairs"] == band_pairs
    return g


SHAPES = [(2, 1), (3, 2), (257, 1), (300, 2), (500, 3), (777, 4), (1000, 7), (1200, 8),
          (900, 16), (1500, 31), (2000, 32), (1000, 64), (1500, 65), (600, 128), (400, 200)]


@pytest.mark.parametrize("n,d", SHAPES)
def test_graph_matches_oracle(orc, n, d):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n * 31 + d)
    eps = float(np.float32(0.12 * math.sqrt(d) if d > 1 else 0.05))
    p = sng.Params(eps=eps, min_pts=4, m=min(150, 3 * n), seed=d)
    xg = torch.from_numpy(x).cuda()
    _compare_graph(orc, x, xg, p, sng)


@pytest.mark.parametrize("n,d,ld", [(500, 3, 4), (500, 3, 3), (700, 5, 9), (300, 64, 72),
                                    (400, 33, 33), (350, 2, 6), (600, 17, 20)])
def test_graph_padded_rows(orc, n, d, ld):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=ld)
    eps = float(np.float32(0.15 * math.sqrt(d)))
    xg, _buf = padded(torch, x, ld)
    assert xg.stride(0) == ld
    p = sng.Params(eps=eps, min_pts=3, m=120, seed=ld + 1)
    _compare_graph(orc, x, xg, p, sng)


COMPILED_SHAPES = [(1, 1), (2, 1), (4, 1), (8, 1), (16, 1), (32, 1), (16, 2), (32, 2), (32, 4),
                   (32, 8), (1, 2), (1, 4), (8, 2), (4, 4), (2, 8), (4, 2), (8, 4), (16, 4),
                   (4, 8), (2, 4)]


@pytest.mark.parametrize("group,nch", COMPILED_SHAPES)
@pytest.mark.parametrize("unroll", [1, 2, 4, 8])
def test_mapping_overrides_agree(orc, group, nch, unroll):
    """Every compiled lanes-per-pair / chunks / batches-in-flight mapping gives
    the oracle's graph (rows one element short of the mapping's width, and
    the full width)."""
    torch, sng = need_gpu()
    d = group * nch * 4 - (1 if unroll % 2 else 0)
    n = 600
    x = datagen.random_points(n, d, seed=group * 10 + nch)
    xg, _buf = padded(torch, x, ((d + 4) // 4) * 4)   # padded, rows stay 16-byte aligned
    p = sng.Params(eps=float(np.float32(0.12 * math.sqrt(d))), min_pts=4, m=150, seed=9,
                   map_group=group, map_unroll=unroll)
    _compare_graph(orc, x, xg, p, sng)


def _compare_cluster(orc, x_np, xg, p, sng):
    n = x_np.shape[0]
    m = p.draws(n)
    labels, core, st = sng.cluster(xg, p, want_core=True)
    r = orc.cluster(x_np, p.eps, p.seed, m, p.min_pts, deg_mode=p.degree_mode,
                    sample_all=p.sample_mode == 1, band_rel=BAND_F32)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    for k in ("kept_edges", "band_pairs", "band_points", "cores", "clusters", "noise"):
        assert st[k] == r[k], (k, st[k], r[k])
    assert st["queries"] == n * m
    return labels, st


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("d,metric", [(16, 0), (32, 0), (64, 0), (128, 0), (64, 2), (128, 1)])
def test_full_row_and_general_kernels_agree(orc, dtype, d, metric):
    """Rows exactly lanes x chunks x vector wide run the full-row kernel
    (packed FP32x2 arithmetic, no bounds tests); unroll 1 has no full-row
    instantiation, so the same mapping then runs the general kernel.  Both
    graphs must equal the oracle's bit for bit."""
    torch, sng = need_gpu()
    n = 3000
    x = datagen.random_points(n, d, seed=d + metric) - (0.5 if metric else 0.0)
    x = np.ascontiguousarray(x, dtype=np.float32)
    if metric:
        xn = x.astype(np.float64)
        s = (xn[:500] * xn[500:1000]).sum(1)
        if metric == 2:
            s /= np.linalg.norm(xn[:500], axis=1) * np.linalg.norm(xn[500:1000], axis=1)
        eps = float(np.float32(np.quantile(s, 0.97)))
    else:
        eps = float(np.float32(0.12 * math.sqrt(d)))
    if dtype == "bf16":
        bits = datagen.bf16_round(x)
        xo = datagen.bf16_to_f32(bits)
        xg = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
        master, band = torch.from_numpy(xo).cuda(), BAND_BF16
    else:
        xo, xg, master, band = x, torch.from_numpy(x).cuda(), None, BAND_F32
    rp, col, bpairs, _ = orc.build_rows(xo, eps, 5, 200, band_rel=band, metric=metric)
    graphs = []
    # the similarity form has no unroll-1 instantiation: there both runs
    # are full-row kernels, checked against the oracle all the same
    for unroll in ((1, 2, 4) if metric == 0 else (2, 4)):
        p = sng.Params(eps=eps, min_pts=3, m=200, seed=5, metric=metric, map_unroll=unroll)
        g = sng.build_graph(xg, p, x_master=master)
        np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
        np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
        assert g["stats"]["band_pairs"] == bpairs
        graphs.append(g)
    vec = 4 if dtype == "f32" else 8
    st = graphs[-1]["stats"]
    assert st["map_group"] * st["map_nch"] * st["map_vec"] == d   # a full-row mapping
    assert st["map_vec"] == vec


@pytest.mark.parametrize("n,d,m,mp", [(2, 1, 1, 1), (50, 2, 49, 2), (3000, 2, 60, 3),
                                      (5000, 3, 100, 4), (4000, 8, 200, 6), (3000, 64, 300, 10),
                                      (2500, 128, 128, 8)])
@pytest.mark.parametrize("deg_mode", [0, 1, 2])
def test_cluster_matches_oracle(orc, n, d, m, mp, deg_mode):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d)
    eps = float(np.float32(0.1 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=mp, m=m, seed=n, degree_mode=deg_mode)
    _compare_cluster(orc, x, torch.from_numpy(x).cuda(), p, sng)


@pytest.mark.parametrize("n,d,m", [(2, 1, 5), (40, 2, 200), (1000, 3, 300), (3000, 16, 100)])
def test_simple_degree_graph(orc, n, d, m):
    """Distinct-neighbour degrees (repeated draws and both directions of a
    pair count once) equal the oracle's; m > n forces many repeats."""
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + 3 * d)
    eps = float(np.float32(0.3 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=3, m=m, seed=n, degree_mode=2)
    _compare_graph(orc, x, torch.from_numpy(x).cuda(), p, sng)


def test_simple_degree_cluster_edges(orc):
    """Steps 3-5 from an edge list with the simple-graph degree: degrees come
    from the edges (deg not passed), including repeats, both directions and a
    self pair, which the oracle counts once."""
    torch, sng = need_gpu()
    n = 500
    rng = np.random.default_rng(4)
    src = rng.integers(0, n, size=4000).astype(np.int32)
    col = rng.integers(0, n, size=4000).astype(np.int32)
    src = np.concatenate([src, src[:300], col[:200], [7]]).astype(np.int32)
    col = np.concatenate([col, col[:300], src[:200], [7]]).astype(np.int32)
    order = np.argsort(src, kind="stable")
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    p = sng.Params(eps=1.0, min_pts=17, m=1, degree_mode=2)
    labels, core, st = sng.cluster_edges(n, torch.from_numpy(src[order]).cuda(),
                                         torch.from_numpy(col[order]).cuda(), None, p,
                                         want_core=True)
    r = orc.cluster_graph(n, rp, col[order], 17, deg_mode=2)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    assert 0 < r["core"].sum() < n


def test_config_small_2d_mixture(orc):
    """n = 10,000 points in d = 2 (95% from 5 Gaussians, 5% uniform), s = 0.01,
    eps = 0.03, MinPts = 3, seed 0: every label equal to the oracle's."""
    torch, sng = need_gpu()
    x = datagen.mixture_2d(10_000, seed=0)
    p = sng.Params(eps=0.03, min_pts=3, s=0.01, seed=0)
    assert p.draws(10_000) == 100
    labels, st = _compare_cluster(orc, x, torch.from_numpy(x).cuda(), p, sng)
    assert st["clusters"] >= 1


@pytest.mark.parametrize("seed,n,d,m_db", [(0, 400, 2, 3), (1, 600, 3, 4), (2, 300, 8, 2)])
def test_sample_all_equals_textbook_dbscan(orc, seed, n, d, m_db):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=seed)
    eps = float(np.float32(0.08 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=2 * (m_db - 1), sample_mode=1)
    labels, st = sng.cluster(torch.from_numpy(x).cuda(), p)
    bl, _ = orc.dbscan_bruteforce(x, eps, m_db)
    np.testing.assert_array_equal(labels.cpu().numpy(), bl)
    # simple-graph degree counts each neighbour once: MinPts = min_samples - 1
    p2 = sng.Params(eps=eps, min_pts=m_db - 1, sample_mode=1, degree_mode=2)
    labels2, _ = sng.cluster(torch.from_numpy(x).cuda(), p2)
    np.testing.assert_array_equal(labels2.cpu().numpy(), bl)


def test_integer_grid_ties_at_eps(orc):
    """Small-integer points put many pairs exactly at eps (d2 == eps^2): the
    closed ball keeps them, on both sides."""
    torch, sng = need_gpu()
    x = datagen.random_points(4000, 3, seed=8, kind="grid")
    p = sng.Params(eps=2.0, min_pts=6, m=300, seed=3)
    labels, st = _compare_cluster(orc, x, torch.from_numpy(x).cuda(), p, sng)
    assert st["band_pairs"] > 0 and st["band_points"] > 0


def test_degenerate_all_noise_and_single_cluster(orc):
    torch, sng = need_gpu()
    x = datagen.random_points(3000, 4, seed=2)
    xg = torch.from_numpy(x).cuda()
    labels, st = sng.cluster(xg, sng.Params(eps=1e-6, min_pts=2, m=50, seed=1))
    assert (labels.cpu().numpy() == -1).all() and st["kept_edges"] == 0 and st["clusters"] == 0
    labels, st = _compare_cluster(orc, x, xg, sng.Params(eps=10.0, min_pts=2, m=50, seed=1), sng)
    assert (labels.cpu().numpy() == 0).all() and st["clusters"] == 1


def test_duplicate_points(orc):
    """All points identical: every draw is kept at distance 0."""
    torch, sng = need_gpu()
    x = np.ones((1000, 5), dtype=np.float32)
    labels, st = _compare_cluster(orc, x, torch.from_numpy(x).cuda(),
                                  sng.Params(eps=1e-3, min_pts=3, m=40, seed=4), sng)
    assert st["kept_edges"] == 40_000


def test_nonfinite_coordinates(orc):
    """NaN and inf rows never pass the eps-test (on both sides)."""
    torch, sng = need_gpu()
    x = datagen.random_points(2000, 3, seed=6)
    x[5] = np.nan
    x[17, 1] = np.inf
    x[18, 2] = -np.inf
    _compare_cluster(orc, x, torch.from_numpy(x).cuda(),
                     sng.Params(eps=0.2, min_pts=4, m=200, seed=6), sng)


def test_repeat_calls_identical():
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(20_000, 16, seed=1)).cuda()
    p = sng.Params(eps=0.3, min_pts=5, m=100, seed=2)
    a, _ = sng.cluster(x, p)
    b, _ = sng.cluster(x, p)
    assert torch.equal(a, b)


def test_ari_kernel_matches_oracle(orc):
    torch, sng = need_gpu()
    rng = np.random.default_rng(0)
    for n in (2, 10, 5000, 200_000):
        a = rng.integers(-1, max(1, n // 7), size=n).astype(np.int32)
        b = np.where(rng.uniform(size=n) < 0.8, a, rng.integers(-1, n, size=n)).astype(np.int32)
        got = sng.ari(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
        assert abs(got - orc.ari(a, b)) < 1e-9


@pytest.mark.parametrize("passes", [2, 3, 7])
@pytest.mark.parametrize("n,d,group", [(3000, 64, 0), (2000, 128, 0), (2500, 32, 0),
                                       (1800, 100, 16), (4000, 24, 8)])
def test_l2_blocked_gather_matches_oracle(orc, passes, n, d, group):
    """The multi-pass (L2-blocked) gather gives the single-pass graph and the
    oracle's, in both degree modes."""
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=passes * 100 + d)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    for deg_mode in (0, 1):
        p = sng.Params(eps=eps, min_pts=4, m=300, seed=passes, map_passes=passes,
                       map_group=group, degree_mode=deg_mode)
        _compare_graph(orc, x, torch.from_numpy(x).cuda(), p, sng)
    labels, st = _compare_cluster(orc, x, torch.from_numpy(x).cuda(),
                                  sng.Params(eps=eps, min_pts=4, m=300, seed=passes,
                                             map_passes=passes, map_group=group), sng)


@pytest.mark.parametrize("n,d,dtype", [(3000, 64, "f32"), (2000, 128, "f32"), (2500, 128, "bf16"),
                                       (1500, 32, "f32"), (1800, 20, "f32")])
def test_prefetch_on_off_same_graph(orc, n, d, dtype):
    """The bulk L2 prefetch of partner rows changes no result."""
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    xg = torch.from_numpy(x).cuda()
    master = None
    if dtype == "bf16":
        bits = datagen.bf16_round(x)
        master = torch.from_numpy(datagen.bf16_to_f32(bits)).cuda()
        xg = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    outs = []
    for flags in (0, sng.SNG_FLAG_PREFETCH):
        p = sng.Params(eps=eps, min_pts=4, m=400, seed=3, flags=flags)
        g = sng.build_graph(xg, p, x_master=master)
        outs.append((g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    if dtype == "f32":
        rp, col, _, _ = orc.build_rows(x, eps, 3, 400, band_rel=BAND_F32)
        np.testing.assert_array_equal(outs[0][1], col)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 16])
def test_lane_per_row_graph_matches_oracle(orc, dtype, d):
    """Rows of at most 4 vectors and enough of them (n = 400,000) run one lane
    per source row; m = 40 leaves a partial keep-bit word per row.  The
    graph equals the oracle's and the warp-per-row kernel's
    (SNG_FLAG_WARP_ROWS), and the labels agree."""
    torch, sng = need_gpu()
    n, m = 400_000, 40
    x = datagen.random_points(n, d, seed=d + 50)
    eps = float(np.float32(0.02 * math.sqrt(d) if d > 1 else 0.0005))
    if dtype == "bf16":
        bits = datagen.bf16_round(x)
        xo = datagen.bf16_to_f32(bits)
        xg = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
        master, band = torch.from_numpy(xo).cuda(), BAND_BF16
    else:
        xo, xg, master, band = x, torch.from_numpy(x).cuda(), None, BAND_F32
    rp, col, bpairs, _ = orc.build_rows(xo, eps, 3, m, band_rel=band)
    assert col.size > 0
    for flags in (0, sng.SNG_FLAG_WARP_ROWS):
        p = sng.Params(eps=eps, min_pts=2, m=m, seed=3, flags=flags)
        g = sng.build_graph(xg, p, x_master=master)
        np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
        np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
        np.testing.assert_array_equal(g["deg"].cpu().numpy(), orc.degrees(n, rp, col))
        assert g["stats"]["band_pairs"] == bpairs
        assert g["stats"]["map_group"] == 1
    r = orc.cluster(xo, eps, 3, m, 2, band_rel=band)
    labels, _ = sng.cluster(xg, sng.Params(eps=eps, min_pts=2, m=m, seed=3), x_master=master)
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])


@pytest.mark.parametrize("form", ["plain", "mma", "fp8"])
def test_no_sync_form_matches_and_replays_as_a_cuda_graph(orc, form):
    """SNG_FLAG_NO_SYNC: the same labels and counters as the synchronous call,
    and the call captured once in a CUDA graph replays correctly, also after
    the points are overwritten in place (n = 10,000 mixture, s = 0.01) -- with
    the plain gather and through the tensor-core screens (their copy, queue
    and open-pair kernel inside the graph)."""
    torch, sng = need_gpu()
    n = 10_000
    x = datagen.mixture_2d(n, seed=0)
    flags = {"plain": 0, "mma": sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA,
             "fp8": sng.SNG_FLAG_SCREEN8}[form]
    p = sng.Params(eps=0.03, min_pts=3, s=0.01, seed=0, flags=flags)
    xg = torch.from_numpy(x).cuda()
    ref, st = sng.cluster(xg, p)
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    counters = torch.zeros(9, dtype=torch.int64, device="cuda")
    sng.cluster_async(xg, p, labels, counters)
    torch.cuda.synchronize()
    assert torch.equal(labels, ref)
    c = counters.cpu().tolist()
    assert c == [0, st["band_pairs"], st["recheck_pairs"], st["band_points"], st["cores"],
                 st["clusters"], st["noise"], st["kept_edges"], 0]
    assert (st["map_screen"] > 0) == (form != "plain")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        sng.cluster_async(xg, p, labels, counters)      # warm-up off the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sng.cluster_async(xg, p, labels, counters)
    labels.fill_(-7)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(labels, ref)
    x2 = datagen.mixture_2d(n, seed=1)
    xg.copy_(torch.from_numpy(x2))
    graph.replay()
    torch.cuda.synchronize()
    r = orc.cluster(x2, 0.03, 0, 100, 3, band_rel=BAND_F32)
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    assert counters[7].item() == r["kept_edges"]


def test_no_sync_form_rejections():
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(300, 3, seed=0)).cuda()
    labels = torch.empty(300, dtype=torch.int32, device="cuda")
    with pytest.raises(sng.SngError) as e:     # distinct-neighbour degree
        sng.cluster_async(x, sng.Params(eps=0.2, min_pts=3, m=20, degree_mode=2), labels)
    assert e.value.status == sng.SNG_EINVAL
    with pytest.raises(sng.SngError) as e:     # phase timing with the flag
        c = sng.Params(eps=0.2, min_pts=3, m=20).to_c(300, 3, 3, sng.SNG_F32)
        c.flags = sng.SNG_FLAG_NO_SYNC | sng.SNG_FLAG_TIMING
        sng._check(sng.lib().sng_cluster(x.data_ptr(), sng.ctypes.byref(c), labels.data_ptr(),
                                         None, None, None))
    assert e.value.status == sng.SNG_EINVAL
    # stats requested with the flag
    p = sng.Params(eps=0.2, min_pts=3, m=20, flags=sng.SNG_FLAG_NO_SYNC)
    with pytest.raises(sng.SngError) as e:
        sng.cluster(x, p)
    assert e.value.status == sng.SNG_EINVAL


@pytest.mark.parametrize("pinned", [False, True])
def test_host_buffer_call_matches_device_call(orc, pinned):
    """sng_cluster_host: host points in (pinned or pageable, FP32 and BF16 with
    a host FP32 master), host labels and core mask out, equal to the device
    call; 80 MB of points so the copy is split over several streams."""
    torch, sng = need_gpu()
    n, d = 1_250_000, 16
    x = datagen.random_points(n, d, seed=21)
    p = sng.Params(eps=float(np.float32(0.05)), min_pts=4, m=30, seed=2)
    ref, ref_core, _ = sng.cluster(torch.from_numpy(x).cuda(), p, want_core=True)
    xt = torch.from_numpy(x)
    if pinned:
        xt = xt.pin_memory()
    labels, core, st = sng.cluster_host(xt, p, want_core=True)
    np.testing.assert_array_equal(labels, ref.cpu().numpy())
    np.testing.assert_array_equal(core, ref_core.cpu().numpy())
    assert st["queries"] == n * 30
    # BF16 storage with the FP32 master on the host
    bits = datagen.bf16_round(x)
    xb = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16)
    xq = torch.from_numpy(datagen.bf16_to_f32(bits))
    if pinned:
        xb, xq = xb.pin_memory(), xq.pin_memory()
    lb, _ = sng.cluster_host(xb, p, x_master=xq)
    ref_b, _ = sng.cluster(xb.cuda(), p, x_master=xq.cuda())
    np.testing.assert_array_equal(lb, ref_b.cpu().numpy())


def test_lane_per_row_every_pair(orc):
    """Every pair queried (s = 1) at n = 80,000 in d = 3 runs one lane per
    row: the graph equals the warp-per-row kernel's, and 150 sampled rows
    equal the oracle's (its full n^2 pass would take too long)."""
    torch, sng = need_gpu()
    n = 80_000
    x = datagen.random_points(n, 3, seed=77)
    eps = float(np.float32(0.01))
    xg = torch.from_numpy(x).cuda()
    graphs = [sng.build_graph(xg, sng.Params(eps=eps, min_pts=3, sample_mode=1, flags=f))
              for f in (0, sng.SNG_FLAG_WARP_ROWS)]
    for k in ("row_ptr", "col", "deg"):
        assert torch.equal(graphs[0][k], graphs[1][k]), k
    rp = graphs[0]["row_ptr"].cpu().numpy()
    col = graphs[0]["col"].cpu().numpy()
    assert col.size > n
    rows = np.sort(np.random.default_rng(3).choice(n, 150, replace=False))
    orp, ocol, _, _ = orc.build_rows(x, eps, 0, n - 1, sample_all=True, rows=rows,
                                     band_rel=BAND_F32)
    for t, i in enumerate(rows):
        np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], ocol[orp[t]:orp[t + 1]])
