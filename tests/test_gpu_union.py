"""Steps 3-4 (components of the core points, Algorithm 1) on graph shapes
that stress the union passes -- streaming hook rounds, compression, and the
union-find pass after them -- against the oracle's steps 3-5 on the same
edge list: long paths whose indices increase along them (the hook rounds
build one chain as long as the path) or run in random order, stars, a
complete bipartite block, many small components, edges listed in both
directions and repeated, and non-core ends.  Each case also has a time
bound far above its expected cost, so a walk that degenerates to quadratic
work fails instead of passing slowly."""
import time

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _run(orc, sng, torch, n, src, col, min_pts, seconds=5.0):
    src = np.asarray(src, dtype=np.int32)
    col = np.asarray(col, dtype=np.int32)
    order = np.argsort(src, kind="stable")
    src, col = src[order], col[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src.astype(np.int64) + 1, 1)
    rp = np.cumsum(rp)
    deg = orc.degrees(n, rp, col, mode=0).astype(np.int32)
    p = sng.Params(eps=1.0, min_pts=min_pts, m=1)
    args = (torch.from_numpy(src).cuda(), torch.from_numpy(col).cuda(),
            torch.from_numpy(deg).cuda())
    sng.cluster_edges(n, *args, p)   # warm-up (module load)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    labels, core, st = sng.cluster_edges(n, *args, p, want_core=True)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < seconds
    r = orc.cluster_graph(n, rp, col, min_pts, deg_mode=0)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    assert st["clusters"] == r["clusters"]
    return r


@pytest.mark.parametrize("n", [200_000, 1_000_000])
def test_sorted_path_is_one_component(orc, n):
    """0-1-2-...: every point hooks to its predecessor, one chain of n."""
    torch, sng = need_gpu()
    a = np.arange(n - 1)
    r = _run(orc, sng, torch, n, a, a + 1, 1)
    assert r["clusters"] == 1


def test_reversed_and_shuffled_paths(orc):
    torch, sng = need_gpu()
    n = 300_000
    rng = np.random.default_rng(1)
    a = np.arange(n - 1)
    rev = _run(orc, sng, torch, n, a + 1, a, 1)          # edges point downwards
    assert rev["clusters"] == 1
    perm = rng.permutation(n)
    r = _run(orc, sng, torch, n, perm[:-1], perm[1:], 1)   # path in random index order
    assert r["clusters"] == 1


def test_stars_bipartite_and_small_components(orc):
    torch, sng = need_gpu()
    n = 400_000
    rng = np.random.default_rng(2)
    src, col = [], []
    # 200 stars of 500 leaves, centre at a random index, leaves pointing in
    centres = rng.choice(n, 200, replace=False)
    rest = np.setdiff1d(np.arange(n), centres)
    rng.shuffle(rest)
    for k, c in enumerate(centres):
        leaves = rest[k * 500:(k + 1) * 500]
        src.append(leaves)
        col.append(np.full(leaves.size, c))
    used = 200 * 500
    # a complete bipartite block 300 x 300 (90,000 edges)
    left, right = rest[used:used + 300], rest[used + 300:used + 600]
    used += 600
    src.append(np.repeat(left, 300))
    col.append(np.tile(right, 300))
    # many pairs and triangles
    small = rest[used:used + 60_000].reshape(-1, 3)
    src += [small[:, 0], small[:, 1]]
    col += [small[:, 1], small[:, 2]]
    src, col = np.concatenate(src), np.concatenate(col)
    # every edge again in the other direction, and 10% repeated
    rep = rng.choice(src.size, src.size // 10, replace=False)
    src2 = np.concatenate([src, col, src[rep]])
    col2 = np.concatenate([col, src, col[rep]])
    r = _run(orc, sng, torch, n, src2, col2, 1)
    assert r["clusters"] == 200 + 1 + 20_000


def test_non_core_ends_split_components(orc):
    """min_pts 3 on a path: interior points have degree 2 (not core) unless
    an extra edge lifts them, so the cores form many short runs joined only
    through border points, which steps 3-4 must not merge."""
    torch, sng = need_gpu()
    n = 200_000
    rng = np.random.default_rng(3)
    a = np.arange(n - 1)
    lift = rng.choice(n, n // 3, replace=False)
    other = rng.integers(0, n, size=lift.size)
    src = np.concatenate([a, lift])
    col = np.concatenate([a + 1, other])
    r = _run(orc, sng, torch, n, src, col, 3)
    assert 1 < r["clusters"] < n
