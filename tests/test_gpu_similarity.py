"""GPU parity of the similarity form of step 2 (inner product or cosine
similarity >= threshold in place of the Euclidean ball) against the FP64
oracle: CSR, degrees, band counts and labels bit-exact for FP32 inputs (each
pair's FP32 value is certified by its own error bound, the rest recomputed in
FP64 in the oracle's order), over row widths that select every vector width
and group size of the default mapping rule, padded rows, exact ties, zero and
non-finite rows, and BF16 storage with a BF16-valued master."""
import math

import numpy as np
import pytest

from gpu_util import BAND_BF16, BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu

DOT, COS = 1, 2


def _threshold(x, metric, q, seed=0):
    """A float32 threshold at quantile q of the similarities of random pairs."""
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    i = rng.integers(0, n, 20000)
    j = rng.integers(0, n, 20000)
    a, b = x[i].astype(np.float64), x[j].astype(np.float64)
    s = (a * b).sum(axis=1)
    if metric == COS:
        s = s / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1) + 1e-300)
    return float(np.float32(np.quantile(s, q)))


def _compare(orc, sng, torch, x, xg, p, band=BAND_F32, master=None, x_oracle=None):
    n = x.shape[0]
    m = p.draws(n)
    xo = x if x_oracle is None else x_oracle
    g = sng.build_graph(xg, p, x_master=master)
    rp, col, band_pairs, _ = orc.build_rows(xo, p.eps, p.seed, m,
                                            sample_all=p.sample_mode == 1, band_rel=band,
                                            metric=p.metric)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    np.testing.assert_array_equal(g["deg"].cpu().numpy(),
                                  orc.degrees(n, rp, col, mode=p.degree_mode))
    assert g["stats"]["band_pairs"] == band_pairs
    labels, core, st = sng.cluster(xg, p, x_master=master, want_core=True)
    r = orc.cluster(xo, p.eps, p.seed, m, p.min_pts, deg_mode=p.degree_mode,
                    sample_all=p.sample_mode == 1, band_rel=band, metric=p.metric)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    for k in ("kept_edges", "band_pairs", "band_points", "cores", "clusters", "noise"):
        assert st[k] == r[k], (k, st[k], r[k])
    return st


SHAPES = [(300, 1), (500, 3), (777, 4), (1000, 7), (1200, 8), (900, 16), (1500, 31),
          (2000, 32), (1000, 64), (1500, 65), (600, 128), (400, 200)]


@pytest.mark.parametrize("metric", [DOT, COS])
@pytest.mark.parametrize("n,d", SHAPES)
def test_similarity_graph_and_labels_match_oracle(orc, metric, n, d):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d) - 0.5
    tau = _threshold(x, metric, 0.97, seed=d)
    p = sng.Params(eps=tau, min_pts=3, m=min(150, 3 * n), seed=d, metric=metric)
    st = _compare(orc, sng, torch, x, torch.from_numpy(np.ascontiguousarray(x)).cuda(), p)
    assert st["kept_edges"] > 0


@pytest.mark.parametrize("metric", [DOT, COS])
@pytest.mark.parametrize("d,ld,fill", [(3, 4, float("nan")), (5, 8, 7.0), (64, 72, float("inf")),
                                       (30, 33, float("nan"))])
def test_padded_rows_ignore_padding(orc, metric, d, ld, fill):
    """Row padding holding NaN / inf / junk must not reach the inner product."""
    torch, sng = need_gpu()
    n = 800
    x = datagen.random_points(n, d, seed=ld) - 0.5
    buf = torch.full((n, ld), fill, dtype=torch.float32, device="cuda")
    buf[:, :d] = torch.from_numpy(x).cuda()
    xg = buf[:, :d]
    tau = _threshold(x, metric, 0.95)
    p = sng.Params(eps=tau, min_pts=3, m=100, seed=5, metric=metric)
    _compare(orc, sng, torch, x, xg, p)


def test_dot_exact_ties_are_kept(orc):
    """Small-integer coordinates put many inner products exactly at the
    (integer) threshold: >= keeps every one, as in the oracle."""
    torch, sng = need_gpu()
    rng = np.random.default_rng(2)
    n, d = 2000, 4
    x = rng.integers(-3, 4, (n, d)).astype(np.float32)
    p = sng.Params(eps=4.0, min_pts=5, m=200, seed=1, metric=DOT)
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    parts = orc.partners(1, n, 0, n, 200)
    at_tau = sum(int((x[parts[i]] @ x[i] == 4.0).sum()) for i in range(n))
    assert at_tau > 1000 and st["band_pairs"] == at_tau


def test_cosine_zero_and_nonfinite_rows(orc):
    """Zero rows are similar to nothing; rows with NaN or inf are decided in
    FP64 exactly as the oracle decides them."""
    torch, sng = need_gpu()
    n, d = 1500, 16
    x = datagen.random_points(n, d, seed=9) - 0.5
    x[::7] = 0.0
    x[3, 2] = np.nan
    x[11, 0] = np.inf
    x[13, 5] = -np.inf
    p = sng.Params(eps=0.3, min_pts=3, m=200, seed=2, metric=COS)
    _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    g = sng.build_graph(torch.from_numpy(x).cuda(), p)
    rp, col = g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()
    assert rp[1] - rp[0] == 0                       # row 0 is a zero row
    assert not np.isin(col, np.arange(0, n, 7)).any()


@pytest.mark.parametrize("tau", [-0.2, 0.0, 0.3])
def test_cosine_extreme_magnitudes(orc, tau):
    """Rows whose FP32 squared norm overflows (entries ~1e20) or underflows
    (~1e-25) have finite FP64 cosines; the FP32 screen must not certify them
    (its reciprocal norms are 0 or inf there), so FP64 decides each pair."""
    torch, sng = need_gpu()
    n, d = 1200, 8
    x = datagen.random_points(n, d, seed=12) - 0.5
    x[::5] *= np.float32(1e20)
    x[1::5] *= np.float32(1e-25)
    p = sng.Params(eps=tau, min_pts=3, m=150, seed=4, metric=COS)
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["kept_edges"] > 0


@pytest.mark.parametrize("metric", [DOT, COS])
@pytest.mark.parametrize("deg_mode", [0, 1, 2])
def test_similarity_degree_modes_and_sample_all(orc, metric, deg_mode):
    torch, sng = need_gpu()
    n, d = 500, 6
    x = datagen.random_points(n, d, seed=4) - 0.5
    tau = _threshold(x, metric, 0.9)
    for p in (sng.Params(eps=tau, min_pts=4, m=300, seed=3, metric=metric, degree_mode=deg_mode),
              sng.Params(eps=tau, min_pts=4, sample_mode=1, metric=metric,
                         degree_mode=deg_mode)):
        _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)


@pytest.mark.parametrize("group", [2, 4, 8, 16, 32])
def test_similarity_mapping_overrides_agree(orc, group):
    torch, sng = need_gpu()
    n, d = 1500, 64
    x = datagen.random_points(n, d, seed=group) - 0.5
    tau = _threshold(x, COS, 0.97)
    for unroll in (2, 4):
        p = sng.Params(eps=tau, min_pts=3, m=120, seed=group, metric=COS, map_group=group,
                       map_unroll=unroll)
        _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)


@pytest.mark.parametrize("n,d", [(3000, 128), (2000, 64), (1200, 5)])
def test_bf16_cosine_exact_when_master_is_bf16(orc, n, d):
    torch, sng = need_gpu()
    x = datagen.sphere_embeddings(n, d, 20, 0.05, seed=d) if d >= 64 else \
        datagen.random_points(n, d, seed=d) - 0.5
    bits = datagen.bf16_round(x)
    xb = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    xq = datagen.bf16_to_f32(bits)
    tau = _threshold(xq, COS, 0.97)
    p = sng.Params(eps=tau, min_pts=4, m=200, seed=d, metric=COS)
    _compare(orc, sng, torch, xq, xb, p, band=BAND_BF16,
             master=torch.from_numpy(xq).cuda(), x_oracle=xq)


def test_similarity_rejected_where_not_supported():
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(200, 3, seed=0)).cuda()
    for p in (sng.Params(eps=0.5, min_pts=3, m=10, metric=5),
              sng.Params(eps=0.5, min_pts=3, m=10, metric=COS, map_passes=2),
              sng.Params(eps=float("nan"), min_pts=3, m=10, metric=DOT)):
        with pytest.raises(sng.SngError) as e:
            sng.cluster(x, p)
        assert e.value.status == sng.SNG_EINVAL
    # a negative threshold is a valid similarity threshold
    labels, _ = sng.cluster(x, sng.Params(eps=-0.25, min_pts=3, m=10, metric=DOT))
    assert labels.numel() == 200


# ---------------------------------------------------------------------------
# The similarity form through the tensor-core screens (a BF16 or FP8 copy of
# the FP32 points, each pair certified from the copy's inner product and the
# rows' own rounding-error bounds, the rest decided in FP64): the same graph,
# band counts and labels as the oracle.

SCREENS = {"mma": 2, "fp8": 4}


def _screen_flags(sng, form):
    return (sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA) if form == "mma" \
        else sng.SNG_FLAG_SCREEN8


@pytest.mark.parametrize("form", sorted(SCREENS))
@pytest.mark.parametrize("metric", [DOT, COS])
@pytest.mark.parametrize("n,d", [(500, 3), (1000, 7), (900, 16), (2000, 32), (1000, 64),
                                 (1500, 65), (600, 128)])
def test_screened_similarity_matches_oracle(orc, form, metric, n, d):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=n + d) - 0.5
    tau = _threshold(x, metric, 0.97, seed=d)
    p = sng.Params(eps=tau, min_pts=3, m=min(150, 3 * n), seed=d, metric=metric,
                   flags=_screen_flags(sng, form))
    st = _compare(orc, sng, torch, x, torch.from_numpy(np.ascontiguousarray(x)).cuda(), p)
    assert st["kept_edges"] > 0 and st["map_screen"] == SCREENS[form]


@pytest.mark.parametrize("form", sorted(SCREENS))
def test_screened_similarity_wider_rows_run_unscreened(orc, form):
    """Past 128 values per row the similarity form reads the FP32 rows."""
    torch, sng = need_gpu()
    x = datagen.random_points(400, 200, seed=3) - 0.5
    tau = _threshold(x, COS, 0.97)
    p = sng.Params(eps=tau, min_pts=3, m=120, seed=3, metric=COS, flags=_screen_flags(sng, form))
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["map_screen"] == 0


@pytest.mark.parametrize("form", sorted(SCREENS))
def test_screened_dot_exact_ties(orc, form):
    torch, sng = need_gpu()
    rng = np.random.default_rng(2)
    n, d = 2000, 4
    x = rng.integers(-3, 4, (n, d)).astype(np.float32)
    p = sng.Params(eps=4.0, min_pts=5, m=200, seed=1, metric=DOT, flags=_screen_flags(sng, form))
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["band_pairs"] > 1000


@pytest.mark.parametrize("form", sorted(SCREENS))
def test_screened_cosine_zero_and_nonfinite_rows(orc, form):
    torch, sng = need_gpu()
    n, d = 1500, 16
    x = datagen.random_points(n, d, seed=9) - 0.5
    x[::7] = 0.0
    x[3, 2] = np.nan
    x[11, 0] = np.inf
    x[13, 5] = -np.inf
    p = sng.Params(eps=0.3, min_pts=3, m=200, seed=2, metric=COS, flags=_screen_flags(sng, form))
    _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)


@pytest.mark.parametrize("form", sorted(SCREENS))
@pytest.mark.parametrize("tau", [-0.2, 0.0, 0.3])
def test_screened_cosine_extreme_magnitudes(orc, form, tau):
    torch, sng = need_gpu()
    n, d = 1200, 8
    x = datagen.random_points(n, d, seed=12) - 0.5
    x[::5] *= np.float32(1e20)
    x[1::5] *= np.float32(1e-25)
    p = sng.Params(eps=tau, min_pts=3, m=150, seed=4, metric=COS, flags=_screen_flags(sng, form))
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["kept_edges"] > 0


@pytest.mark.parametrize("form", sorted(SCREENS))
@pytest.mark.parametrize("metric", [DOT, COS])
def test_screened_similarity_degree_modes_and_sample_all(orc, form, metric):
    torch, sng = need_gpu()
    n, d = 500, 6
    x = datagen.random_points(n, d, seed=4) - 0.5
    tau = _threshold(x, metric, 0.9)
    for deg_mode in (0, 1, 2):
        for p in (sng.Params(eps=tau, min_pts=4, m=300, seed=3, metric=metric,
                             degree_mode=deg_mode, flags=_screen_flags(sng, form)),
                  sng.Params(eps=tau, min_pts=4, sample_mode=1, metric=metric,
                             degree_mode=deg_mode, flags=_screen_flags(sng, form))):
            _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)


@pytest.mark.parametrize("form", sorted(SCREENS))
def test_screened_cosine_embeddings_leave_few_pairs_open(orc, form):
    """Unit vectors around 100 centres (the embedding workload's recipe at
    4*10^4 points, d = 128): the same graph and labels as the oracle, and
    the screen certifies all but a small share of the pairs."""
    torch, sng = need_gpu()
    n, d = 40_000, 128
    x = datagen.sphere_embeddings(n, d, 100, 0.0375, seed=1)
    p = sng.Params(eps=float(np.float32(1 - 0.6 ** 2 / 2)), min_pts=8, m=200, seed=1,
                   metric=COS, flags=_screen_flags(sng, form))
    st = _compare(orc, sng, torch, x, torch.from_numpy(x).cuda(), p)
    assert st["kept_edges"] > 0 and st["screen_pairs"] < 0.05 * n * 200
