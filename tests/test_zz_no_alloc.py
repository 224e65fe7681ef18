"""The entry point that allocates nothing (sng_cluster_noalloc).

It exists for callers that cannot allocate device memory when they cluster:
a plugin whose host application reserved all device memory up front, or a
real-time loop that cannot accept cudaMalloc's device synchronisation or its
failure under memory pressure.  It must give exactly what sng_cluster gives
on the same input -- and what the oracle's Algorithm 1 gives -- call after
call, although every call reuses the same fixed scratch array (which keeps
the previous call's contents), and after its first call on a device it must
not change the device's free memory.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import ctypes
import math

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _noalloc_into(sng, torch, x, p, labels):
    n, d, ld = x.shape[0], x.shape[1], x.stride(0)
    st = sng.sng_stats()
    rc = sng.lib().sng_cluster_noalloc(x.data_ptr(), ctypes.byref(p.to_c(n, d, ld, sng.SNG_F32)),
                                       labels.data_ptr(), ctypes.byref(st),
                                       torch.cuda.current_stream().cuda_stream)
    return rc, st.as_dict()


def _noalloc(sng, torch, x, p):
    labels = torch.full((x.shape[0],), -7, dtype=torch.int32, device="cuda")
    rc, st = _noalloc_into(sng, torch, x, p, labels)
    return rc, labels, st


def test_noalloc_matches_sng_cluster_on_two_calls_in_a_row(orc):
    torch, sng = need_gpu()
    xs, off = datagen.point_clouds(2, seed=12, n_min=30_000, n_max=60_000)
    for b, seed in ((0, 5), (1, 6)):
        host = np.ascontiguousarray(xs[off[b]:off[b + 1]])
        buf = torch.from_numpy(host).cuda()
        x = buf[:, :3]                       # d = 3 in 16-byte rows
        p = sng.Params(eps=0.3, min_pts=4, m=96, seed=seed)
        ref, ref_st = sng.cluster(x, p)
        want = orc.cluster(host[:, :3], p.eps, seed, 96, 4, band_rel=BAND_F32)
        np.testing.assert_array_equal(ref.cpu().numpy(), want["labels"])
        for flags in (0, sng.SNG_FLAG_WARP_ROWS):
            q = sng.Params(eps=0.3, min_pts=4, m=96, seed=seed, flags=flags)
            for _ in range(2):
                rc, labels, st = _noalloc(sng, torch, x, q)
                assert rc == sng.SNG_OK, sng.last_error()
                assert torch.equal(labels, ref)
                for k in ("kept_edges", "cores", "clusters", "noise", "band_pairs"):
                    assert st[k] == ref_st[k], k
                assert st["kept_edges"] == want["kept_edges"]


@pytest.mark.parametrize("d", [8, 32, 64])
def test_noalloc_wider_rows_match_sng_cluster_and_oracle(orc, d):
    """Rows of 8, 32 and 64 values (16-byte aligned) run with 4, 8 or 16 lanes
    per pair by default, twice in a row, equal to sng_cluster and the oracle."""
    torch, sng = need_gpu()
    n = 20_000
    x = datagen.random_points(n, d, seed=d)
    xg = torch.from_numpy(x).cuda()
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=64, seed=d)
    ref, ref_st = sng.cluster(xg, p)
    want = orc.cluster(x, eps, d, 64, 4, band_rel=BAND_F32)
    np.testing.assert_array_equal(ref.cpu().numpy(), want["labels"])
    for _ in range(2):
        rc, labels, st = _noalloc(sng, torch, xg, p)
        assert rc == sng.SNG_OK, sng.last_error()
        assert torch.equal(labels, ref)
        assert st["kept_edges"] == ref_st["kept_edges"] == want["kept_edges"]


def test_noalloc_leaves_free_device_memory_unchanged():
    """After the first call on the device (which loads the entry point's code
    and its fixed array), further calls change no free device memory."""
    torch, sng = need_gpu()
    n, d = 30_000, 3
    x = torch.from_numpy(datagen.random_points(n, d, seed=3)).cuda()
    p = sng.Params(eps=0.1, min_pts=4, m=64, seed=3)
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    rc, _ = _noalloc_into(sng, torch, x, p, labels)
    assert rc == sng.SNG_OK, sng.last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rc, _ = _noalloc_into(sng, torch, x, p, labels)
        assert rc == sng.SNG_OK, sng.last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, sng = need_gpu()
    x = torch.zeros((400_000, 4), device="cuda")[:, :3]
    rc, _, _ = _noalloc(sng, torch, x, sng.Params(eps=0.3, min_pts=4, m=512, seed=1))
    assert rc == sng.SNG_EINVAL
    assert "scratch" in sng.last_error()


def test_noalloc_rejects_simple_degree():
    torch, sng = need_gpu()
    x = torch.zeros((1000, 3), device="cuda")
    rc, _, _ = _noalloc(sng, torch, x, sng.Params(eps=0.3, min_pts=4, m=16, degree_mode=2))
    assert rc == sng.SNG_EINVAL
