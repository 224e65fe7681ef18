"""Sharding independent clouds across ranks (one process per GPU).

Clouds in the batched form share nothing, so N ranks split them with no
data-path collective: rank r takes a contiguous range of clouds whose sampled
query counts (n_b * m_b) sum to about 1/N of the total, and clusters it with
its own plan.  Labels are cloud-local, so a rank's output needs no
renumbering.
"""
from __future__ import annotations

import numpy as np


def cloud_queries(offsets, m_per_cloud=None, m: int | None = None, s: float | None = None):
    sizes = np.diff(np.asarray(offsets, dtype=np.int64))
    if m_per_cloud is not None:
        mb = np.asarray(m_per_cloud, dtype=np.int64)
    elif m is not None:
        mb = np.full(sizes.size, int(m), dtype=np.int64)
    else:
        mb = np.ceil(float(s) * sizes).astype(np.int64)
    return sizes * mb


def shard_clouds(offsets, rank: int, world: int, m_per_cloud=None, m=None, s=None):
    """Clouds [b0, b1) of this rank, balanced by sampled queries."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    q = cloud_queries(offsets, m_per_cloud, m, s)
    cum = np.concatenate([[0], np.cumsum(q)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")))
    cuts.append(q.size)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, q.size))
    return int(cuts[rank]), int(cuts[rank + 1])


def local_offsets(offsets, b0: int, b1: int):
    """Offsets of clouds b0..b1-1 relative to the rank's first row."""
    o = np.asarray(offsets, dtype=np.int64)[b0:b1 + 1]
    return o - o[0]
