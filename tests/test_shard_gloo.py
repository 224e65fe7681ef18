"""Multi-rank path on CPU: two gloo ranks split independent clouds by query
count and each clusters its own shard (the oracle stands in for the GPU here);
rank 0 gathers the shards and checks they cover every cloud exactly once with
the single-process result."""
import os
import socket

import numpy as np
import pytest

from paper_2006_06743_gb300 import datagen
from paper_2006_06743_gb300.shard import cloud_queries, local_offsets, shard_clouds


def test_shards_cover_and_balance():
    x, off = datagen.point_clouds(37, seed=2, n_min=50, n_max=5000)
    q = cloud_queries(off, m=40)
    for world in (1, 2, 3, 8):
        ranges = [shard_clouds(off, r, world, m=40) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == 37
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0
        loads = [q[a:b].sum() for a, b in ranges]
        assert max(loads) <= q.sum() / world + q.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, result_path):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, off = datagen.point_clouds(9, seed=4, n_min=100, n_max=700)
    b0, b1 = shard_clouds(off, rank, world, m=30)
    lo = local_offsets(off, b0, b1)
    xs = x[off[b0]:off[b1], :3]
    labels = np.empty(xs.shape[0], np.int32)
    for k in range(b1 - b0):
        xb = np.ascontiguousarray(xs[lo[k]:lo[k + 1]])
        labels[lo[k]:lo[k + 1]] = oracle.cluster(xb, 0.4, 7 + b0 + k, 30, 3)["labels"]
    got = [None] * world
    dist.all_gather_object(got, (b0, b1, labels))
    if rank == 0:
        full = np.concatenate([g[2] for g in sorted(got, key=lambda g: g[0])])
        np.save(result_path, full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path, orc):
    mp = pytest.importorskip("torch.multiprocessing")
    path = str(tmp_path / "labels.npy")
    mp.start_processes(_worker, args=(2, _free_port(), path), nprocs=2, start_method="spawn")
    full = np.load(path)
    x, off = datagen.point_clouds(9, seed=4, n_min=100, n_max=700)
    want = np.concatenate([
        orc.cluster(np.ascontiguousarray(x[off[b]:off[b + 1], :3]), 0.4, 7 + b, 30, 3)["labels"]
        for b in range(9)])
    np.testing.assert_array_equal(full, want)
