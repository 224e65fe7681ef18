"""Batched form: many independent clouds in one persistent launch must give,
cloud by cloud, the labels of Algorithm 1 on that cloud alone (the oracle, and
the single-cloud GPU call), with cloud b using seed base + b."""
import ctypes

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _run_batched(sng, torch, x, offsets, p, m_per_cloud=None, plan=False, repeats=1):
    xg = torch.from_numpy(x).cuda()
    labels = torch.full((x.shape[0],), -7, dtype=torch.int32, device="cuda")
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    mp = None if m_per_cloud is None else np.ascontiguousarray(m_per_cloud, dtype=np.int64)
    cp = p.to_c(0, 3, x.shape[1], sng.SNG_F32)
    st = sng.sng_stats()
    L = sng.lib()
    if not plan:
        rc = L.sng_cluster_batched(xg.data_ptr(), off.ctypes.data, len(off) - 1,
                                   ctypes.byref(cp), mp.ctypes.data if mp is not None else None,
                                   labels.data_ptr(), ctypes.byref(st),
                                   torch.cuda.current_stream().cuda_stream)
        sng._check(rc)
        return labels.cpu().numpy(), st.as_dict(), []
    h = ctypes.c_void_p()
    sng._check(L.sng_batch_plan_create(off.ctypes.data, len(off) - 1, ctypes.byref(cp),
                                       mp.ctypes.data if mp is not None else None,
                                       ctypes.byref(h)))
    outs = []
    try:
        for _ in range(repeats):
            labels.fill_(-7)
            sng._check(L.sng_batch_run(h, xg.data_ptr(), labels.data_ptr(), ctypes.byref(st),
                                       torch.cuda.current_stream().cuda_stream))
            outs.append(labels.cpu().numpy())
    finally:
        L.sng_batch_plan_destroy(h)
    return outs[-1], st.as_dict(), outs


@pytest.mark.parametrize("use_plan", [False, True])
@pytest.mark.parametrize("lanes", [False, True])
def test_batched_matches_oracle_per_cloud(orc, use_plan, lanes):
    """Lane per row (the default for float4 rows) and warp per row
    (SNG_FLAG_WARP_ROWS): m = 40 puts a partial keep-bit word at the end of
    every row."""
    torch, sng = need_gpu()
    x, off = datagen.point_clouds(12, seed=3, n_min=200, n_max=3000)
    p = sng.Params(eps=0.3, min_pts=4, m=40, seed=100,
                   flags=0 if lanes else sng.SNG_FLAG_WARP_ROWS)
    labels, st, _ = _run_batched(sng, torch, x, off, p, plan=use_plan)
    tot = dict(cores=0, clusters=0, noise=0, kept_edges=0)
    for b in range(len(off) - 1):
        xb = np.ascontiguousarray(x[off[b]:off[b + 1], :3])
        r = orc.cluster(xb, p.eps, p.seed + b, p.m, p.min_pts, band_rel=BAND_F32)
        np.testing.assert_array_equal(labels[off[b]:off[b + 1]], r["labels"], err_msg=f"cloud {b}")
        for k in tot:
            tot[k] += r[k]
    for k, v in tot.items():
        assert st[k] == v, k


def test_batched_per_cloud_draws_and_s_rule(orc):
    torch, sng = need_gpu()
    x, off = datagen.point_clouds(6, seed=4, n_min=100, n_max=900)
    sizes = np.diff(off)
    mpc = np.array([1, 5, 33, 64, 65, 200])
    p = sng.Params(eps=0.4, min_pts=3, seed=7)
    labels, _, _ = _run_batched(sng, torch, x, off, p, m_per_cloud=mpc)
    for b in range(len(sizes)):
        xb = np.ascontiguousarray(x[off[b]:off[b + 1], :3])
        r = orc.cluster(xb, p.eps, p.seed + b, int(mpc[b]), p.min_pts, band_rel=BAND_F32)
        np.testing.assert_array_equal(labels[off[b]:off[b + 1]], r["labels"])
    # s-rule: m_b = ceil(s * n_b)
    p2 = sng.Params(eps=0.4, min_pts=3, seed=7, s=0.05)
    labels, _, _ = _run_batched(sng, torch, x, off, p2)
    for b in range(len(sizes)):
        xb = np.ascontiguousarray(x[off[b]:off[b + 1], :3])
        r = orc.cluster(xb, p2.eps, p2.seed + b, p2.draws(int(sizes[b])), p2.min_pts,
                        band_rel=BAND_F32)
        np.testing.assert_array_equal(labels[off[b]:off[b + 1]], r["labels"])


def test_batched_graph_replay_identical_and_matches_single_calls():
    torch, sng = need_gpu()
    x, off = datagen.point_clouds(40, seed=5, n_min=500, n_max=6000)
    p = sng.Params(eps=0.3, min_pts=4, m=200, seed=11, map_tile=256)
    last, _, outs = _run_batched(sng, torch, x, off, p, plan=True, repeats=3)
    for o in outs:
        np.testing.assert_array_equal(o, last)
    for b in (0, 17, 39):
        xb = torch.from_numpy(np.ascontiguousarray(x[off[b]:off[b + 1], :3])).cuda()
        lb, _ = sng.cluster(xb, sng.Params(eps=p.eps, min_pts=p.min_pts, m=p.m, seed=p.seed + b))
        np.testing.assert_array_equal(lb.cpu().numpy(), last[off[b]:off[b + 1]])


def test_batched_lane_rows_per_cloud_draws_and_modes(orc):
    """Lane per row with per-cloud draw counts (1 .. 200), out-degree, every
    pair queried, and each compiled unroll; rows of d = 3 padded to 4 with
    NaN in the padding, which must not reach the distance."""
    torch, sng = need_gpu()
    x, off = datagen.point_clouds(6, seed=8, n_min=100, n_max=900)
    x = x.copy()
    x[:, 3] = np.nan
    mpc = np.array([1, 5, 33, 64, 65, 200])
    for unroll in (2, 4):
        for deg_mode in (0, 1):
            p = sng.Params(eps=0.4, min_pts=3, seed=7, map_unroll=unroll, degree_mode=deg_mode)
            labels, _, _ = _run_batched(sng, torch, x, off, p, m_per_cloud=mpc)
            for b in range(len(off) - 1):
                xb = np.ascontiguousarray(x[off[b]:off[b + 1], :3])
                r = orc.cluster(xb, p.eps, p.seed + b, int(mpc[b]), p.min_pts, deg_mode=deg_mode,
                                band_rel=BAND_F32)
                np.testing.assert_array_equal(labels[off[b]:off[b + 1]], r["labels"])
    p = sng.Params(eps=0.4, min_pts=3, sample_mode=1)
    labels, _, _ = _run_batched(sng, torch, x, off, p)
    for b in range(len(off) - 1):
        xb = np.ascontiguousarray(x[off[b]:off[b + 1], :3])
        r = orc.cluster(xb, p.eps, 0, int(off[b + 1] - off[b]) - 1, p.min_pts, sample_all=True,
                        band_rel=BAND_F32)
        np.testing.assert_array_equal(labels[off[b]:off[b + 1]], r["labels"])


@pytest.mark.parametrize("unroll,block,tile", [(1, 256, 1024), (2, 128, 64), (8, 256, 4096)])
def test_batched_mappings_agree(unroll, block, tile):
    torch, sng = need_gpu()
    x, off = datagen.point_clouds(20, seed=6, n_min=300, n_max=5000)
    ref, _, _ = _run_batched(sng, torch, x, off, sng.Params(eps=0.3, min_pts=4, m=64, seed=1))
    got, _, _ = _run_batched(sng, torch, x, off,
                             sng.Params(eps=0.3, min_pts=4, m=64, seed=1, map_unroll=unroll,
                                        map_block=block, map_tile=tile))
    np.testing.assert_array_equal(got, ref)


def test_batched_rejects_bad_tables():
    torch, sng = need_gpu()
    x = np.zeros((10, 4), dtype=np.float32)
    p = sng.Params(eps=0.3, min_pts=4, m=8)
    for off in ([0, 1, 10], [1, 5, 10], [0, 5, 4]):
        with pytest.raises(sng.SngError) as e:
            _run_batched(sng, torch, x, np.array(off), p)
        assert e.value.status == sng.SNG_EINVAL
    # the simple-graph degree needs a pair set per cloud: not in this form
    with pytest.raises(sng.SngError) as e:
        _run_batched(sng, torch, x, np.array([0, 5, 10]),
                     sng.Params(eps=0.3, min_pts=4, m=8, degree_mode=2))
    assert e.value.status == sng.SNG_EINVAL
