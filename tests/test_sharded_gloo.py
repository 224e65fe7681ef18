"""One dataset across ranks (the multi-GPU form of the plain path), run on
CPU with gloo and world size 2: each rank builds the sampled graph of its
source rows, degrees are all-reduced, kept edges all-gathered, and steps 3-5
run on the whole edge list.  The oracle stands in for the GPU kernels; the
exchange code is the one GPU ranks run.  Labels, cores and the edge list must
equal the single-process oracle's."""
import os
import socket

import numpy as np
import pytest

from paper_2006_06743_gb300 import datagen
from paper_2006_06743_gb300.distributed import LocalGraph, cluster_sharded, row_range

N, D, M, EPS, MINPTS, SEED = 3000, 3, 60, 0.05, 4, 7


class OracleCompute:
    """Oracle-backed stand-in for GpuCompute (CPU tensors)."""

    def __init__(self, x, deg_mode=0):
        self.x = x
        self.deg_mode = deg_mode
        self.simple_degree = deg_mode == 2

    def local_graph(self, lo, hi):
        import torch
        import oracle
        rows = np.arange(lo, hi, dtype=np.int64)
        rp, col, _, _ = oracle.build_rows(self.x, EPS, SEED, M, rows=rows)
        src = np.repeat(rows, np.diff(rp)).astype(np.int32)
        deg = np.zeros(self.x.shape[0], dtype=np.int64)
        np.add.at(deg, src, 1)       # out-degree of this rank's rows
        np.add.at(deg, col, 1)       # in-degree they give their partners
        return LocalGraph(torch.from_numpy(src), torch.from_numpy(col.astype(np.int32)),
                          torch.from_numpy(deg.astype(np.int32)))

    def cluster_edges(self, n, src, col, deg):
        import oracle
        s, c = src.numpy(), col.numpy()
        order = np.argsort(s, kind="stable")
        rp = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rp, s + 1, 1)
        rp = np.cumsum(rp)
        r = oracle.cluster_graph(n, rp, c[order], MINPTS, deg_mode=self.deg_mode)
        if deg is None:
            assert self.simple_degree     # simple degrees come from the edges
        else:
            np.testing.assert_array_equal(r["deg"], deg.numpy())   # all-reduced degrees
        return r["labels"], r["core"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out, deg_mode=0):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = datagen.random_points(N, D, seed=SEED)
    labels, core, (src, col) = cluster_sharded(OracleCompute(x, deg_mode), N)
    np.savez(f"{out}.{rank}.npz", labels=labels, core=core, src=src.numpy(), col=col.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_row_ranges_cover_rows():
    for n in (1, 7, 1000):
        for world in (1, 2, 3, 8):
            r = [row_range(n, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))


@pytest.mark.parametrize("world,deg_mode", [(2, 0), (3, 0), (2, 2)])
def test_sharded_ranks_match_single_process(tmp_path, orc, world, deg_mode):
    """deg_mode 2 (distinct neighbours) skips the degree all-reduce: every rank
    counts degrees from the gathered edge list."""
    mp = pytest.importorskip("torch.multiprocessing")
    out = str(tmp_path / "res")
    mp.start_processes(_worker, args=(world, _free_port(), out, deg_mode), nprocs=world,
                       start_method="spawn")
    x = datagen.random_points(N, D, seed=SEED)
    want = orc.cluster(x, EPS, SEED, M, MINPTS, deg_mode=deg_mode)
    rp, col, _, _ = orc.build_rows(x, EPS, SEED, M)
    for r in range(world):
        got = np.load(f"{out}.{r}.npz")
        np.testing.assert_array_equal(got["labels"], want["labels"])
        np.testing.assert_array_equal(got["core"], want["core"])
        np.testing.assert_array_equal(got["col"], col)
        np.testing.assert_array_equal(got["src"], np.repeat(np.arange(N), np.diff(rp)))
