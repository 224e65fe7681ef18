"""SNG-DBSCAN on one dataset across several GPUs (one process per GPU).

Algorithm 1's step 2 is independent per source point, so ranks split the
source rows: with the points replicated on every rank, rank r draws the
partners of rows [n r / N, n (r+1) / N) and keeps its edges.  Step 3 needs
every point's degree and the whole core subgraph, so the ranks exchange

  * degrees: each rank's partial degrees (its draws' out- and in-degree
    contributions) are summed with one all-reduce of n int32;
  * edges: the kept draws (source, partner) are all-gathered; contiguous row
    ranges in rank order make the concatenation the graph's CSR order;

after which every rank runs steps 3-5 on the full edge list and holds the
same labels.  With the simple-graph degree (distinct neighbours) partial
degrees do not add up across ranks (two ranks may draw the same pair), so
the all-reduce is skipped and each rank counts degrees from the gathered
edge list.  The exchange is written once against a small compute
interface, so the CPU test (gloo, oracle as compute) runs the same code as
GPU ranks (NCCL, libsng.so as compute).
"""
from __future__ import annotations

from dataclasses import dataclass


def row_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous source rows of a rank (balanced to within one row)."""
    return n * rank // world, n * (rank + 1) // world


@dataclass
class LocalGraph:
    src: object        # int32 tensor [E_r]: source row of every kept draw
    col: object        # int32 tensor [E_r]: partner, draw order within a row
    deg: object        # int32 tensor [n]: this rank's degree contributions


class GpuCompute:
    """Compute on this rank's GPU through libsng.so."""

    def __init__(self, x, params, x_master=None):
        self.x, self.params, self.x_master = x, params, x_master
        self.simple_degree = params.degree_mode == 2
        self.last_stats = None      # stats of the last local graph (phase times)

    def local_graph(self, lo: int, hi: int) -> LocalGraph:
        import torch

        from . import Params, build_graph
        p = Params(**{**self.params.__dict__, "row_begin": lo, "row_end": hi})
        if lo == hi:   # an empty shard still contributes zero degrees
            n = self.x.shape[0]
            z = torch.zeros(0, dtype=torch.int32, device=self.x.device)
            return LocalGraph(z, z.clone(), torch.zeros(n, dtype=torch.int32,
                                                        device=self.x.device))
        g = build_graph(self.x, p, x_master=self.x_master)
        self.last_stats = g["stats"]
        rp = g["row_ptr"]
        counts = rp[lo + 1:hi + 1] - rp[lo:hi]
        rows = torch.arange(lo, hi, device=rp.device, dtype=torch.int32)
        src = torch.repeat_interleave(rows, counts)
        return LocalGraph(src, g["col"], g["deg"])

    def cluster_edges(self, n: int, src, col, deg):
        from . import cluster_edges
        labels, core, st = cluster_edges(n, src, col, deg, self.params, want_core=True)
        return labels, core


def cluster_sharded(compute, n: int, group=None):
    """Steps 2-5 with step 2 split across the ranks of ``group``.  Returns
    (labels, core, edges) on every rank (identical on all ranks)."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    lo, hi = row_range(n, rank, world)
    g = compute.local_graph(lo, hi)
    dev = g.deg.device
    deg = None
    if not getattr(compute, "simple_degree", False):
        deg = g.deg.clone()
        dist.all_reduce(deg, op=dist.ReduceOp.SUM, group=group)
    # all-gather the edge lists (padded to the longest; sizes first)
    e = torch.tensor([g.src.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(e) for _ in range(world)]
    dist.all_gather(sizes, e, group=group)
    sizes = [int(s.item()) for s in sizes]
    emax = max(sizes)
    pair = torch.full((2, emax), -1, dtype=torch.int32, device=dev)
    pair[0, :g.src.numel()] = g.src
    pair[1, :g.col.numel()] = g.col
    parts = [torch.empty_like(pair) for _ in range(world)]
    dist.all_gather(parts, pair, group=group)
    src = torch.cat([parts[r][0, :sizes[r]] for r in range(world)]).contiguous()
    col = torch.cat([parts[r][1, :sizes[r]] for r in range(world)]).contiguous()
    labels, core = compute.cluster_edges(n, src, col, deg)
    return labels, core, (src, col)
