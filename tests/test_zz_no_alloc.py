"""The entry point that allocates nothing (sng_cluster_noalloc).

It exists for callers that cannot allocate device memory when they cluster:
a plugin whose host application reserved all device memory up front, or a
real-time loop that cannot accept cudaMalloc's device synchronisation or its
failure under memory pressure.  It must give exactly what sng_cluster gives
on the same input, call after call, although every call reuses the same fixed
scratch array (which keeps the previous call's contents).

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _noalloc(sng, torch, x, p):
    n, d, ld = x.shape[0], x.shape[1], x.stride(0)
    labels = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st = sng.sng_stats()
    rc = sng.lib().sng_cluster_noalloc(x.data_ptr(), ctypes.byref(p.to_c(n, d, ld, sng.SNG_F32)),
                                       labels.data_ptr(), ctypes.byref(st),
                                       torch.cuda.current_stream().cuda_stream)
    return rc, labels, st.as_dict()


def test_noalloc_matches_sng_cluster_on_two_calls_in_a_row():
    torch, sng = need_gpu()
    xs, off = datagen.point_clouds(2, seed=12, n_min=30_000, n_max=60_000)
    for b, seed in ((0, 5), (1, 6)):
        buf = torch.from_numpy(np.ascontiguousarray(xs[off[b]:off[b + 1]])).cuda()
        x = buf[:, :3]                       # d = 3 in 16-byte rows
        p = sng.Params(eps=0.3, min_pts=4, m=96, seed=seed)
        ref, ref_st = sng.cluster(x, p)
        for _ in range(2):
            rc, labels, st = _noalloc(sng, torch, x, p)
            assert rc == sng.SNG_OK, sng.last_error()
            assert torch.equal(labels, ref)
            for k in ("kept_edges", "cores", "clusters", "noise", "band_pairs"):
                assert st[k] == ref_st[k], k


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
