"""The C ABI on the CPU: the library builds, loads and exports every symbol
include/sng.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sng.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sng_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_boundary():
    names = _declared()
    for want in ("sng_build_graph", "sng_cluster", "sng_cluster_batched", "sng_graph_free",
                 "sng_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_2006_06743_gb300 as sng
    sng.build()
    lib = ctypes.CDLL(sng.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(sng.SIGNATURES)


def test_binding_loads_and_reports_without_gpu():
    import paper_2006_06743_gb300 as sng
    sng.build()
    L = sng.lib()
    assert L.sng_strerror(0) == b"ok"
    assert L.sng_strerror(-1) == b"invalid argument"
    assert sng.launch_count() >= 0


def test_invalid_params_rejected_on_host():
    """Validation happens before any CUDA call, so it works without a GPU."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    p = sng.Params(eps=-1.0, min_pts=3, s=0.1).to_c(100, 3, 3, sng.SNG_F32)
    st = sng.sng_stats()
    rc = sng.lib().sng_cluster(ctypes.c_void_p(256), ctypes.byref(p), ctypes.c_void_p(256), None,
                               ctypes.byref(st), None)
    assert rc == sng.SNG_EINVAL
    assert "eps" in sng.last_error()


def _mapping(sng, d, ld, dtype, addr, **kw):
    master = 8192 if dtype == sng.SNG_BF16 else 0
    p = sng.Params(eps=0.5, min_pts=3, m=100, **kw).to_c(1000, d, ld, dtype, master)
    out = (ctypes.c_int32 * 7)()
    rc = sng.lib().sng_gather_mapping(ctypes.c_void_p(addr), ctypes.byref(p), out)
    return rc, list(out)


def test_default_mapping_is_compiled_for_every_shape():
    """The mapping rule must land on a compiled kernel for every row width the
    library accepts, for both element types and every row alignment (no GPU:
    the query only inspects the arguments)."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    checked = 0
    for dtype, dmax, esize in ((sng.SNG_F32, 1024, 4), (sng.SNG_BF16, 2048, 2)):
        for d in list(range(1, 130)) + [255, 256, 257, 500, 512, 1000, 1024, 2000, 2048]:
            for pad in (0, 1, 3, 8):
                ld = d + pad
                for addr in (4096, 4096 + 2 * esize):
                    rc, m = _mapping(sng, d, ld, dtype, addr)
                    if rc != 0:
                        # only rows too wide for the compiled shapes may be refused
                        assert "wider" in sng.last_error(), (dtype, d, ld, addr, sng.last_error())
                        assert d > 256, (dtype, d, ld, addr)
                        continue
                    assert m[6] == 1, (dtype, d, ld, addr, m)
                    checked += 1
        # aligned rows up to the documented maximum always work
        rc, m = _mapping(sng, dmax, dmax, dtype, 4096)
        assert rc == 0 and m[6] == 1
    assert checked > 1500


def test_autotuner_candidates_are_compiled():
    import paper_2006_06743_gb300 as sng
    sng.build()
    for d, dtype in ((64, sng.SNG_F32), (128, sng.SNG_F32), (128, sng.SNG_BF16), (32, sng.SNG_F32),
                     (3, sng.SNG_F32)):
        ld = ((d + 3) // 4) * 4 if dtype == sng.SNG_F32 else ((d + 7) // 8) * 8
        g0 = 1
        n_ok = 0
        for g in (1, 2, 4, 8, 16, 32):
            for u in (1, 2, 4, 8):
                rc, m = _mapping(sng, d, ld, dtype, 4096, map_group=g, map_unroll=u)
                if rc == 0 and m[6] == 1:
                    n_ok += 1
        assert n_ok >= 4


class _FakeCudaRows:
    """Stands in for a CUDA tensor of n x d rows (shape, stride, dtype, device)
    so the autotuner's candidate list can be checked without a GPU."""

    def __init__(self, n, d, dtype):
        import torch
        self.shape = (n, d)
        self.dtype = dtype
        self.is_cuda = True
        self.device = torch.device("cuda", 0)
        self._ld = d

    def stride(self, dim=None):
        return (self._ld, 1) if dim is None else (self._ld, 1)[dim]


def test_autotuner_offers_the_tiled_form_where_it_fits(monkeypatch):
    """Tiled candidates come first for Euclidean hashed draws on point sets
    over 48 MiB whose buckets (~8.4 B per draw) fit in half the free memory;
    their slice counts are the library's rule (two slices in 88 MiB, clamped
    to [2, 32]), half of it and two more; none for small sets, similarity
    metrics, every-pair sampling or too little memory."""
    import torch
    from paper_2006_06743_gb300 import Params, autotune
    free = [200 << 30]
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda dev=None: (free[0], 280 << 30))

    def tiled(n, d, dtype=torch.float32, **kw):
        cands = autotune.candidates(_FakeCudaRows(n, d, dtype), Params(eps=1.0, min_pts=5, **kw))
        cands = [c for c in cands if not c.get("screen")]
        t = [c for c in cands if c.get("tiled")]
        if t:
            first = next(i for i, c in enumerate(cands) if not c.get("tiled"))
            assert first == len(t)                   # tiled candidates lead the list
        return sorted({c["map_tile"] for c in t}), {c["map_unroll"] for c in t}

    # 10^6 x 64 FP32 = 256 MB: rule k = ceil(512 MB / 88 MiB) = 6 -> {6 (as 0), 3, 8}
    ks, us = tiled(1_000_000, 64, s=0.001)
    assert ks == [0, 3, 8] and us == {2, 4}
    # 5e6 x 128 FP32 = 2.56 GB: rule 56 -> clamped to 32 -> {32 (as 0), 16, 32}
    assert tiled(5_000_000, 128, m=1000)[0] == [0, 16, 32]
    # 4e5 x 64 FP32 = 102 MB: rule ceil(204.8 MB / 92.3 MB) = 3 -> {3, 2, 5}
    assert tiled(400_000, 64, m=1000)[0] == [0, 2, 5]
    # small sets, similarity metrics and every-pair sampling: none
    assert tiled(100_000, 64, m=100)[0] == []
    assert tiled(1_000_000, 64, m=1000, metric=2)[0] == []
    assert tiled(200_000, 64, sample_mode=1)[0] == []
    # buckets must fit in half the free memory: 8.4 B x 10^9 draws = 8.4 GB
    # (15 GiB free: half is 8.05 GB; 17 GiB: 9.1 GB)
    free[0] = 15 << 30
    assert tiled(1_000_000, 64, m=1000)[0] == []
    free[0] = 17 << 30
    assert tiled(1_000_000, 64, m=1000)[0] == [0, 3, 8]


def test_autotuner_offers_the_bf16_screen_for_fp32_points(monkeypatch):
    """Screened candidates (SNG_FLAG_SCREEN16) lead the list for FP32 points,
    Euclidean form, hashed draws: the tensor-core forms over the BF16 copy and
    one over the FP8 copy (d <= 128), the direct gather over the BF16 copy with
    the default lanes per pair for 8-value chunks and half of it, and, for
    copies over 48 MiB whose buckets fit, the tiled form with the copy's
    slice count and one more.  For similarity metrics only the tensor-core
    forms; none for BF16 points or every-pair sampling; the flag reaches the
    parameters."""
    import torch
    from paper_2006_06743_gb300 import (SNG_FLAG_SCREEN8, SNG_FLAG_SCREEN16, SNG_FLAG_SCREEN_MMA,
                                        Params, autotune)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda dev=None: (200 << 30, 280 << 30))

    def screened(n, d, dtype=torch.float32, **kw):
        cands = autotune.candidates(_FakeCudaRows(n, d, dtype), Params(eps=1.0, min_pts=5, **kw))
        sc = [c for c in cands if c.get("screen")]
        assert cands[:len(sc)] == sc                 # screened candidates lead the list
        return sc

    sc = screened(1_000_000, 64, s=0.001)
    mma = [c for c in sc if c.get("mma")]        # tensor-core dot products first
    assert sc[:len(mma)] == mma and {c["map_unroll"] for c in mma} == {0, 4, 2}
    assert not any(c.get("mma") for c in screened(1_000_000, 200, m=100))   # d > 128
    fp8 = [c for c in sc if c.get("fp8")]       # one FP8-copy candidate after them
    assert len(fp8) == 1 and sc[len(mma)] == fp8[0]
    assert not any(c.get("fp8") for c in screened(1_000_000, 200, m=100))   # d > 128
    p8 = autotune.apply(Params(eps=1.0, min_pts=5), {"mapping": fp8[0]})
    assert p8.flags & SNG_FLAG_SCREEN8 and not p8.flags & SNG_FLAG_SCREEN_MMA
    direct = [c for c in sc if not c.get("tiled") and not c.get("mma") and not c.get("fp8")]
    tiled = [c for c in sc if c.get("tiled")]
    assert {c["map_group"] for c in direct} == {4, 8} and {c["map_unroll"] for c in direct} == {2, 4}
    # BF16 copy of 10^6 x 64 = 128 MB: ceil(256 MB / 88 MiB) = 3 -> {3, 4}
    assert sorted({c["map_tile"] for c in tiled}) == [3, 4]
    assert {c["map_group"] for c in tiled} == {0, 8}
    p = autotune.apply(Params(eps=1.0, min_pts=5), {"mapping": sc[0]})
    assert p.flags & SNG_FLAG_SCREEN16
    p = autotune.apply(Params(eps=1.0, min_pts=5), {"mapping": sc[0]})
    assert p.flags & SNG_FLAG_SCREEN_MMA and p.flags & SNG_FLAG_SCREEN16
    # small point sets: the direct screened gather only
    assert all(not c.get("tiled") for c in screened(100_000, 64, m=100))
    assert screened(1_000_000, 64, dtype=torch.bfloat16, m=1000) == []
    # similarity metrics: the tensor-core forms only (d <= 128)
    sim = screened(1_000_000, 64, m=1000, metric=2)
    assert sim and all(c.get("mma") or c.get("fp8") for c in sim)
    assert screened(1_000_000, 200, m=1000, metric=2) == []
    assert screened(200_000, 64, sample_mode=1) == []
    # Manhattan / Chebyshev: the pair-kernel gather over the BF16 copy, then
    # over the FP32 points; the latter alone for BF16 points
    for metric in (3, 4):
        two = screened(1_000_000, 64, metric=metric)
        assert len(two) == 1 and not two[0].get("mma") and not two[0].get("fp8")
        all_ = autotune.candidates(_FakeCudaRows(1_000_000, 64, torch.float32),
                                   Params(eps=1.0, min_pts=5, metric=metric))
        assert len(all_) == 2 and not all_[1].get("screen")
        pm = autotune.apply(Params(eps=1.0, min_pts=5, metric=metric), {"mapping": two[0]})
        assert pm.flags & SNG_FLAG_SCREEN16 and not pm.flags & SNG_FLAG_SCREEN_MMA
        one = autotune.candidates(_FakeCudaRows(1_000_000, 64, torch.bfloat16),
                                  Params(eps=1.0, min_pts=5, metric=metric))
        assert len(one) == 1 and not one[0].get("screen")


def test_random_row_probe_rejects_bad_arguments_on_host():
    """The probe validates its sizes before any CUDA call."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    v = ctypes.c_double()
    L = sng.lib()
    assert L.sng_measure_random_rows(1 << 20, 96, 1 << 24, 0, ctypes.byref(v), None) \
        == sng.SNG_EINVAL
    assert "row_bytes" in sng.last_error()
    assert L.sng_measure_random_rows(512, 128, 1 << 24, 0, ctypes.byref(v), None) \
        == sng.SNG_EINVAL
    assert L.sng_measure_random_rows(1 << 27, 128, 1 << 24, 0, ctypes.byref(v), None) \
        == sng.SNG_EINVAL      # 16 GiB of rows
    assert L.sng_measure_random_rows(1 << 20, 128, 100, 0, ctypes.byref(v), None) \
        == sng.SNG_EINVAL
    assert L.sng_measure_random_rows(1 << 20, 128, 1 << 24, 0, None, None) == sng.SNG_EINVAL


_REJECTIONS = [
    # (params overrides, to_c overrides, keyword of the message)
    (dict(), dict(n=1), "n must be"),
    (dict(), dict(d=0), "d must be"),
    (dict(), dict(ld=2), "ld must be"),
    (dict(), dict(dtype=7), "unknown dtype"),
    (dict(degree_mode=5), dict(), "degree_mode"),
    (dict(sample_mode=3), dict(), "sample_mode"),
    (dict(min_pts=0), dict(), "min_pts"),
    (dict(metric=5), dict(), "unknown metric"),
    (dict(eps=float("inf")), dict(), "finite"),
    (dict(eps=1e-20), dict(), "eps must be in"),
    (dict(eps=1e19, metric=3), dict(), "eps must be in"),
    (dict(metric=4), dict(dtype="bf16", master=256), "Manhattan and Chebyshev"),
    (dict(metric=1, map_passes=2), dict(), "one pass"),
    (dict(flags=4 | 1), dict(), "phase timing"),
    (dict(flags=4, degree_mode=2), dict(), "distinct-neighbour"),
    (dict(band_rel=0.5), dict(), "band_rel"),
    (dict(), dict(x=258), "aligned"),
    (dict(), dict(dtype="bf16"), "x_f32_master"),
    (dict(s=0.0, m=0), dict(), "s must be"),
    (dict(m=2 ** 31), dict(), "m must be"),
]


@pytest.mark.parametrize("over,cover,word", _REJECTIONS)
def test_every_parameter_rejection_happens_on_the_host(over, cover, word):
    """Each invalid parameter is reported as SNG_EINVAL with its own message
    before any CUDA call (so without a GPU)."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    kw = dict(eps=0.5, min_pts=3, s=0.1)
    kw.update(over)
    shape = dict(n=100, d=4, ld=4, dtype=sng.SNG_F32, master=0, x=256)
    shape.update(cover)
    if shape["dtype"] == "bf16":
        shape["dtype"] = sng.SNG_BF16
    p = sng.Params(**kw).to_c(shape["n"], shape["d"], shape["ld"], shape["dtype"], shape["master"])
    st = sng.sng_stats()
    rc = sng.lib().sng_cluster(ctypes.c_void_p(shape["x"]), ctypes.byref(p), ctypes.c_void_p(256),
                               None, ctypes.byref(st), None)
    assert rc == sng.SNG_EINVAL
    assert word in sng.last_error(), sng.last_error()


def test_other_entry_points_reject_on_the_host():
    """sng_build_graph, sng_cluster_host, sng_cluster_edges and the L2 probe
    check their own arguments before any CUDA call."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    L = sng.lib()
    ok = sng.Params(eps=0.5, min_pts=3, s=0.1)
    st = sng.sng_stats()
    x = ctypes.c_void_p(256)

    def err(rc, word):
        assert rc == sng.SNG_EINVAL
        assert word in sng.last_error(), sng.last_error()

    # sng_build_graph: no output, the no-sync flag
    p = ok.to_c(100, 4, 4, sng.SNG_F32)
    err(L.sng_build_graph(x, ctypes.byref(p), None, ctypes.byref(st), None), "out is NULL")
    p = sng.Params(eps=0.5, min_pts=3, s=0.1, flags=sng.SNG_FLAG_NO_SYNC).to_c(100, 4, 4,
                                                                           sng.SNG_F32)
    g = sng.sng_graph()
    err(L.sng_build_graph(x, ctypes.byref(p), ctypes.byref(g), ctypes.byref(st), None),
        "SNG_FLAG_NO_SYNC")
    # sng_cluster_host: NULL buffers, the no-sync flag, BF16 without master
    p = ok.to_c(100, 4, 4, sng.SNG_F32)
    err(L.sng_cluster_host(None, ctypes.byref(p), x, None, ctypes.byref(st), None), "NULL")
    p = sng.Params(eps=0.5, min_pts=3, s=0.1, flags=sng.SNG_FLAG_NO_SYNC).to_c(100, 4, 4,
                                                                           sng.SNG_F32)
    err(L.sng_cluster_host(x, ctypes.byref(p), x, None, ctypes.byref(st), None), "synchronises")
    p = ok.to_c(100, 4, 4, sng.SNG_BF16)
    err(L.sng_cluster_host(x, ctypes.byref(p), x, None, ctypes.byref(st), None), "master")
    # sng_cluster_edges: degrees, counts, edge arrays, MinPts
    p = ok.to_c(100, 4, 4, sng.SNG_F32)
    err(L.sng_cluster_edges(100, x, x, 5, None, ctypes.byref(p), x, None, None, None),
        "deg is NULL")
    err(L.sng_cluster_edges(0, x, x, 5, x, ctypes.byref(p), x, None, None, None), "n must be")
    err(L.sng_cluster_edges(100, x, x, -1, x, ctypes.byref(p), x, None, None, None),
        "num_edges")
    err(L.sng_cluster_edges(100, None, x, 5, x, ctypes.byref(p), x, None, None, None),
        "src / col")
    p = sng.Params(eps=0.5, min_pts=0, s=0.1).to_c(100, 4, 4, sng.SNG_F32)
    err(L.sng_cluster_edges(100, x, x, 5, x, ctypes.byref(p), x, None, None, None), "min_pts")
    # the L2 read probe: buffer size and passes
    v = ctypes.c_double()
    err(L.sng_measure_l2_read(1024, 10, ctypes.byref(v), None), "bytes")
    err(L.sng_measure_l2_read(1 << 24, 0, ctypes.byref(v), None), "passes")
    err(L.sng_measure_l2_read(1 << 24, 10, None, None), "gbs is NULL")
