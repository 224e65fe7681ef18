"""The multi-GPU form of the plain path on one GPU: shards of step 2 built
one after another (row ranges), degrees summed, edges concatenated, steps 3-5
through sng_cluster_edges - equal to one sng_cluster call; and the exchange
code itself on a single NCCL rank."""
import os
import socket

import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shards,deg_mode", [(2, 0), (3, 0), (4, 1)])
def test_row_shards_recompose_the_plain_result(shards, deg_mode):
    torch, sng = need_gpu()
    from paper_2006_06743_gb300.distributed import GpuCompute, row_range
    n = 20_000
    x = torch.from_numpy(datagen.random_points(n, 16, seed=3)).cuda()
    p = sng.Params(eps=0.3, min_pts=6, m=120, seed=2, degree_mode=deg_mode)
    ref, ref_core, _ = sng.cluster(x, p, want_core=True)
    full = sng.build_graph(x, p)
    comp = GpuCompute(x, p)
    parts = [comp.local_graph(*row_range(n, r, shards)) for r in range(shards)]
    deg = torch.stack([g.deg for g in parts]).sum(0).to(torch.int32)
    src = torch.cat([g.src for g in parts]).contiguous()
    col = torch.cat([g.col for g in parts]).contiguous()
    assert torch.equal(deg, full["deg"])
    assert torch.equal(col, full["col"])
    labels, core = comp.cluster_edges(n, src, col, deg)
    assert torch.equal(labels, ref)
    assert torch.equal(core, ref_core)


def test_single_rank_nccl_exchange():
    torch, sng = need_gpu()
    import torch.distributed as dist
    from paper_2006_06743_gb300.distributed import GpuCompute, cluster_sharded
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0,
                            world_size=1)
    try:
        n = 30_000
        x = torch.from_numpy(datagen.random_points(n, 8, seed=4)).cuda()
        p = sng.Params(eps=0.25, min_pts=5, m=100, seed=9)
        ref, _ = sng.cluster(x, p)
        labels, core, _ = cluster_sharded(GpuCompute(x, p), n)
        assert torch.equal(labels, ref)
    finally:
        dist.destroy_process_group()


def test_cluster_edges_rejects_out_of_range_edges_without_fault():
    torch, sng = need_gpu()
    n = 100
    src = torch.tensor([0, 1, 2, 150], dtype=torch.int32, device="cuda")
    col = torch.tensor([1, 2, 3, 4], dtype=torch.int32, device="cuda")
    deg = torch.full((n,), 3, dtype=torch.int32, device="cuda")
    with pytest.raises(sng.SngError) as e:
        sng.cluster_edges(n, src, col, deg, sng.Params(eps=1.0, min_pts=2))
    assert e.value.status == sng.SNG_EINTERNAL
    labels, _ = sng.cluster_edges(n, src[:3], col[:3], deg, sng.Params(eps=1.0, min_pts=2))
    assert labels[:4].tolist() == [0, 0, 0, 0]
