"""Pins for the oracle's Algorithm 1 (Section 3): the eps-test, degrees, core
mask, core components and border labels, each checked against hand-worked
cases, textbook DBSCAN (scikit-learn and a brute-force all-pairs version),
exact integer arithmetic, graph-library components and sampling statistics."""
import math

import numpy as np
import pytest

from golden_io import alg1_case
from paper_2006_06743_gb300 import datagen


# ----------------------------------------------------------- hand-worked

@pytest.mark.parametrize("name", ["alg1_line_full_graph.txt", "alg1_border_tie.txt"])
def test_alg1_hand_cases_full_graph(orc, name):
    c = alg1_case(name)
    n = c["x"].shape[0]
    r = orc.cluster(c["x"], c["eps"], seed=0, m=n - 1, min_pts=c["min_pts"], sample_all=True)
    np.testing.assert_array_equal(r["core"], c["core"])
    np.testing.assert_array_equal(r["labels"], c["labels"])
    lab, core = orc.dbscan_bruteforce(c["x"], c["eps"], c["min_pts_db"])
    np.testing.assert_array_equal(core, c["core"])
    np.testing.assert_array_equal(lab, c["labels"])


def _csr(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append(b)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([b for r in rows for b in r], dtype=np.int32)
    return rp, col


def test_hand_graph_path_star_and_isolated(orc):
    # path 0-1-2-3 (out-degree mode: each vertex's own draws), star centred
    # at 5 with leaves 6,7,8 drawing the centre, isolated 9.
    edges = [(0, 1), (1, 0), (1, 2), (2, 1), (2, 3), (3, 2),
             (6, 5), (7, 5), (8, 5), (5, 6)]
    rp, col = _csr(10, edges)
    deg = orc.degrees(10, rp, col, mode=0)
    # undirected multigraph: 0:2 1:4 2:4 3:2 5:4 6:2 7:1 8:1
    np.testing.assert_array_equal(deg, [2, 4, 4, 2, 0, 4, 2, 1, 1, 0])
    np.testing.assert_array_equal(orc.degrees(10, rp, col, mode=1),
                                  [1, 2, 2, 1, 0, 1, 1, 1, 1, 0])
    np.testing.assert_array_equal(orc.degrees(10, rp, col, mode=2),
                                  [1, 2, 2, 1, 0, 3, 1, 1, 1, 0])
    r = orc.cluster_graph(10, rp, col, min_pts=4, deg_mode=0)
    # cores 1, 2, 5; component {1,2} label 1, {5} label 5
    np.testing.assert_array_equal(r["core"], [0, 1, 1, 0, 0, 1, 0, 0, 0, 0])
    np.testing.assert_array_equal(r["labels"], [1, 1, 1, 1, -1, 5, 5, 5, 5, -1])
    assert r["clusters"] == 2 and r["noise"] == 2 and r["cores"] == 3


def test_hand_graph_two_cliques_border_both_directions(orc):
    # cliques {0,1,2} and {4,5,6}; 3 is drawn by 2 (in-edge) and draws 6 (out-edge)
    edges = [(a, b) for a in (0, 1, 2) for b in (0, 1, 2) if a != b]
    edges += [(a, b) for a in (4, 5, 6) for b in (4, 5, 6) if a != b]
    edges += [(2, 3), (3, 6)]
    rp, col = _csr(7, edges)
    r = orc.cluster_graph(7, rp, col, min_pts=4, deg_mode=0)
    np.testing.assert_array_equal(r["core"], [1, 1, 1, 0, 1, 1, 1])
    np.testing.assert_array_equal(r["labels"], [0, 0, 0, 0, 4, 4, 4])
    # drop the in-edge: 3 only reaches {4,5,6} through its own draw
    edges.remove((2, 3))
    rp, col = _csr(7, edges)
    r = orc.cluster_graph(7, rp, col, min_pts=4, deg_mode=0)
    np.testing.assert_array_equal(r["labels"], [0, 0, 0, 4, 4, 4, 4])


def test_noncore_edges_do_not_join_components(orc):
    # 0-1 core pair, 2 non-core bridging to core pair 3-4: two clusters
    edges = [(0, 1), (1, 0), (0, 1), (1, 0), (1, 2), (2, 3), (3, 4), (4, 3), (3, 4), (4, 3)]
    rp, col = _csr(5, edges)
    r = orc.cluster_graph(5, rp, col, min_pts=4, deg_mode=0)
    np.testing.assert_array_equal(r["core"], [1, 1, 0, 1, 1])
    np.testing.assert_array_equal(r["labels"], [0, 0, 0, 3, 3])


# ------------------------------------------------- distances and eps-test

def test_dist2_exact_on_integer_grid(orc):
    rng = np.random.default_rng(3)
    for d in (1, 2, 3, 7, 64, 129):
        a = rng.integers(-50, 50, size=d)
        b = rng.integers(-50, 50, size=d)
        exact = int(((a - b) ** 2).sum())
        assert orc.dist2(a.astype(np.float32), b.astype(np.float32)) == float(exact)


def test_edges_match_integer_arithmetic(orc):
    """On small-integer points every squared distance is an exact integer, so
    the kept set is fixed by integer comparisons alone."""
    n, d, m = 300, 3, 40
    x = datagen.random_points(n, d, seed=11, kind="grid")
    eps = math.sqrt(5.0)
    rp, col, _, _ = orc.build_rows(x, eps, seed=77, m=m)
    p = orc.partners(seed=77, n=n, i0=0, ni=n, m=m)
    xi = x.astype(np.int64)
    d2 = ((xi[:, None, :] - xi[p]) ** 2).sum(-1)
    eps2 = float(np.float32(eps)) ** 2
    keep = d2 <= eps2
    np.testing.assert_array_equal(np.diff(rp), keep.sum(1))
    np.testing.assert_array_equal(col, p[keep])


def test_band_flags(orc):
    """Pairs at exactly eps are in every band; far pairs in none."""
    x = np.array([[0.0], [1.0], [5.0]], dtype=np.float32)
    rp, col, band_pairs, bp = orc.build_rows(x, 1.0, seed=0, m=2, sample_all=True,
                                             band_rel=1e-5)
    assert band_pairs == 2                  # (0,1) drawn from both sides
    np.testing.assert_array_equal(bp, [1, 1, 0])
    np.testing.assert_array_equal(col, [1, 0])


# --------------------------------------- textbook DBSCAN at s = 1

def _sk_dbscan(x, eps, min_samples):
    sk = pytest.importorskip("sklearn.cluster")
    db = sk.DBSCAN(eps=eps, min_samples=min_samples, metric="euclidean",
                   algorithm="brute").fit(x.astype(np.float64))
    core = np.zeros(x.shape[0], dtype=np.uint8)
    core[db.core_sample_indices_] = 1
    return db.labels_, core


@pytest.mark.parametrize("seed,n,d", [(0, 60, 1), (1, 120, 2), (2, 200, 3), (3, 150, 8),
                                      (4, 90, 2), (5, 250, 2)])
@pytest.mark.parametrize("m_db", [2, 3, 5])
def test_sample_all_equals_textbook_dbscan(orc, seed, n, d, m_db):
    """s = 1 (every pair queried) reduces Algorithm 1 to DBSCAN: with the
    undirected multigraph degree, MinPts = 2 (min_samples - 1)."""
    x = datagen.random_points(n, d, seed=seed)
    rng = np.random.default_rng(seed)
    eps = float(np.float32(rng.uniform(0.03, 0.12) * math.sqrt(d)))
    r = orc.cluster(x, eps, seed=0, m=n - 1, min_pts=2 * (m_db - 1), sample_all=True)
    bl, bc = orc.dbscan_bruteforce(x, eps, m_db)
    np.testing.assert_array_equal(r["core"], bc)
    np.testing.assert_array_equal(r["labels"], bl)
    # out-degree mode: MinPts = min_samples - 1
    r1 = orc.cluster(x, eps, seed=0, m=n - 1, min_pts=m_db - 1, deg_mode=1, sample_all=True)
    np.testing.assert_array_equal(r1["labels"], bl)
    # simple-graph degree: distinct neighbours = |N_eps(x)| - 1 as well
    r2 = orc.cluster(x, eps, seed=0, m=n - 1, min_pts=m_db - 1, deg_mode=2, sample_all=True)
    np.testing.assert_array_equal(r2["labels"], bl)
    np.testing.assert_array_equal(r2["deg"], r1["deg"])
    # scikit-learn: same cores; same partition of cores; borders valid
    sl, sc = _sk_dbscan(x, eps, m_db)
    np.testing.assert_array_equal(sc, bc)
    cores = bc.astype(bool)
    assert orc.ari(sl[cores], bl[cores]) == 1.0
    np.testing.assert_array_equal(sl < 0, bl < 0)


def test_simple_degree_counts_distinct_pairs(orc):
    """Distinct-neighbour degree against a set of unordered pairs built in
    Python from hashed draws with many repeats (n = 40, m = 60)."""
    x = datagen.random_points(40, 2, seed=3)
    rp, col, _, _ = orc.build_rows(x, 0.4, 5, 60)
    pairs = set()
    for i in range(40):
        for p in col[rp[i]:rp[i + 1]]:
            pairs.add((min(i, int(p)), max(i, int(p))))
    want = np.zeros(40, dtype=np.int32)
    for a, b in pairs:
        want[a] += 1
        want[b] += 1
    got = orc.degrees(40, rp, col, mode=2)
    np.testing.assert_array_equal(got, want)
    assert (orc.degrees(40, rp, col, mode=0) > got).any()   # repeats were present


# ------------------------------------------------ components cross-checks

def _random_graph(n, e, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=e)
    dst = rng.integers(0, n - 1, size=e)
    dst = dst + (dst >= src)
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp), dst.astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_components_bfs_uf_scipy_agree(orc, seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    n = 400
    rp, col = _random_graph(n, 500 + 60 * seed, seed)
    core = (np.random.default_rng(seed + 100).uniform(size=n) < 0.7).astype(np.uint8)
    cb, kb = orc.components(n, rp, col, core, "bfs")
    cu, ku = orc.components(n, rp, col, core, "uf")
    np.testing.assert_array_equal(cb, cu)
    assert kb == ku
    src = np.repeat(np.arange(n), np.diff(rp))
    keep = core[src].astype(bool) & core[col].astype(bool)
    a = sp.coo_matrix((np.ones(keep.sum()), (src[keep], col[keep])), shape=(n, n))
    ncc, lab = csgraph.connected_components(a, directed=False)
    cidx = np.nonzero(core)[0]
    assert orc.ari(lab[cidx], cb[cidx]) == 1.0
    # component label = smallest member index
    for c in np.unique(cb[cidx]):
        assert c == cidx[cb[cidx] == c].min()
    assert kb == len(np.unique(lab[cidx]))


@pytest.mark.parametrize("seed", range(4))
def test_label_invariants_on_sampled_graph(orc, seed):
    n, d = 2000, 2
    x = datagen.random_points(n, d, seed=seed)
    r = orc.cluster(x, 0.04, seed=seed, m=60, min_pts=4)
    rp, col, _, _ = orc.build_rows(x, 0.04, seed=seed, m=60)
    lab, core = r["labels"], r["core"].astype(bool)
    src = np.repeat(np.arange(n), np.diff(rp))
    # labels constant across every core-core edge
    cc = core[src] & core[col]
    assert (lab[src[cc]] == lab[col[cc]]).all()
    # every core labelled with the smallest core index of its component
    assert (lab[core] >= 0).all()
    for c in np.unique(lab[core]):
        members = np.nonzero(core & (lab == c))[0]
        assert members.min() == c
    # borders: non-core with a label is adjacent to a core of that label,
    # and that label is the smallest among adjacent cores; noise has no core neighbour
    best = np.full(n, np.iinfo(np.int32).max, dtype=np.int64)
    e1 = core[src] & ~core[col]
    np.minimum.at(best, col[e1], lab[src[e1]])
    e2 = ~core[src] & core[col]
    np.minimum.at(best, src[e2], lab[col[e2]])
    nc = ~core
    has = best < np.iinfo(np.int32).max
    assert (lab[nc & has] == best[nc & has]).all()
    assert (lab[nc & ~has] == -1).all()
    # degrees: undirected multigraph sums to twice the kept draws
    assert r["deg"].sum() == 2 * r["kept_edges"]


# ------------------------------------------------------- statistics (Lemma 2)

def test_out_hits_follow_ball_mass(orc):
    """The proof of Lemma 2 treats |N_{n,s}(x, eps)| as a sum of sn Bernoulli
    draws of mean P(B(x, eps)).  For points uniform in the unit cube, interior
    points have P = (4/3) pi eps^3 (up to the n-1 vs n normalisation), so the
    mean out-degree over interior points is m * P within a few standard errors."""
    n, m, eps = 20_000, 400, 0.08
    x = datagen.random_points(n, 3, seed=21, kind="uniform")
    rp, _, _, _ = orc.build_rows(x, eps, seed=4, m=m)
    inner = np.all((x > eps) & (x < 1 - eps), axis=1)
    out = np.diff(rp)[inner]
    p = 4.0 / 3.0 * math.pi * eps ** 3
    mean = out.mean()
    se = math.sqrt(m * p * (1 - p) / inner.sum())
    assert abs(mean - m * p) < 5 * se + 0.01 * m * p, (mean, m * p, se)
    # variance close to binomial (points' own ball masses are all equal here)
    assert 0.7 < out.var() / (m * p * (1 - p)) < 1.3


# ------------------------------------------------- surrogate-gated form

def test_gated_form_reduces_to_plain_and_prefix(orc):
    """With every point ungated the gated form is Algorithm 1 itself; a point
    limited to m_row[i] draws keeps exactly the kept draws among its first
    m_row[i] (prefix of the same stream)."""
    n, m = 1500, 80
    x = datagen.random_points(n, 2, seed=31)
    plain = orc.cluster(x, 0.05, seed=3, m=m, min_pts=4)
    full = orc.cluster_gated(x, 0.05, 3, m, 4, forced=np.zeros(n, np.uint8),
                             m_row=np.full(n, m, np.int32))
    np.testing.assert_array_equal(full["labels"], plain["labels"])
    assert full["queries"] == n * m
    rng = np.random.default_rng(0)
    m_row = rng.integers(0, m + 1, size=n).astype(np.int32)
    rp, col, _, _ = orc.build_rows(x, 0.05, 3, m, m_row=m_row)
    p = orc.partners(3, n, 0, n, m)
    xx = x.astype(np.float64)
    for i in rng.choice(n, 40, replace=False):
        cand = p[i, :m_row[i]]
        d2 = ((xx[i] - xx[cand]) ** 2).sum(1)
        want = cand[d2 <= float(np.float32(0.05)) ** 2]
        np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], want)


def test_gated_forced_core_and_noise(orc):
    # path 0-1-2-3 drawn by 0,1,2 only: degrees 1,2,2,1 (multigraph)
    rp, col = _csr(4, [(0, 1), (1, 2), (2, 3)])
    r = orc.cluster_graph(4, rp, col, min_pts=2)
    np.testing.assert_array_equal(r["labels"], [1, 1, 1, 1])
    # forcing 3 to core makes it a core of the same component
    r = orc.cluster_graph(4, rp, col, min_pts=2, forced=np.array([0, 0, 0, 1], np.uint8))
    np.testing.assert_array_equal(r["core"], [0, 1, 1, 1])
    np.testing.assert_array_equal(r["labels"], [1, 1, 1, 1])
    # forcing 2 to non-core cuts the path: 3 becomes noise, 2 a border of 1
    r = orc.cluster_graph(4, rp, col, min_pts=2, forced=np.array([0, 0, 2, 0], np.uint8))
    np.testing.assert_array_equal(r["core"], [0, 1, 0, 0])
    np.testing.assert_array_equal(r["labels"], [1, 1, 1, -1])


def test_gated_weighted_degrees(orc):
    """Weighted degrees: each kept draw of row i counts w_row[i] at both ends
    (multigraph) or at i only (out-degree); unit weights give the plain
    degrees."""
    rp, col = _csr(4, [(0, 1), (0, 2), (1, 2), (3, 2)])
    r = orc.cluster_graph(4, rp, col, min_pts=1, w_row=np.ones(4, np.int32))
    np.testing.assert_array_equal(r["deg"], orc.degrees(4, rp, col, 0))
    w = np.array([16, 64, 16, 32], np.int32)
    r = orc.cluster_graph(4, rp, col, min_pts=64, w_row=w)
    # deg: 0 -> 16+16, 1 -> 16 (in from 0) + 64 (own), 2 -> 16+64+32, 3 -> 32
    np.testing.assert_array_equal(r["deg"], [32, 80, 112, 32])
    np.testing.assert_array_equal(r["core"], [0, 1, 1, 0])
    r = orc.cluster_graph(4, rp, col, min_pts=32, deg_mode=1, w_row=w)
    np.testing.assert_array_equal(r["deg"], [32, 64, 0, 32])


@pytest.mark.parametrize("openmp", [False, True])
@pytest.mark.parametrize("block", [1, 97, 5000, 100_000])
def test_row_blocks_equal_one_call(orc, openmp, block):
    """The CPU baseline's row-block driver (plain and OpenMP builds of the same
    source) gives exactly the one-call step-2 graph."""
    n, d, m = 5000, 8, 40
    x = datagen.random_points(n, d, seed=block)
    eps = float(np.float32(0.12 * math.sqrt(d)))
    rp, col, bp, _ = orc.build_rows(x, eps, 11, m)
    rp2, col2, bp2 = orc.build_rows_blocks(x, eps, 11, m, block=block, openmp=openmp)
    np.testing.assert_array_equal(rp2, rp)
    np.testing.assert_array_equal(col2, col)
    assert bp2 == bp
    assert orc.threads(openmp) >= 1
    # a leading range of rows: the first rows of the same graph
    rp3, col3, _ = orc.build_rows_blocks(x, eps, 11, m, block=block, openmp=openmp, n_rows=1234)
    np.testing.assert_array_equal(rp3, rp[:1235])
    np.testing.assert_array_equal(col3, col[:rp[1234]])


def test_gate_rule_hand_cases(orc):
    """The gate's rule (thresholds, draw budgets, degree weights) against the
    hand-worked rows of tests/golden/gate_rule.txt, one point at a time and
    all points of one setting together."""
    from golden_io import read_rows
    rows = read_rows("gate_rule.txt")
    groups = {}
    for r in rows:
        key = tuple(r[:6])
        groups.setdefault(key, []).append(r[6:])
        m, pn, pc, cf, nf, rw = int(r[0]), float(r[1]), float(r[2]), float(r[3]), float(r[4]), \
            bool(int(r[5]))
        forced, m_row, w_row = orc.gate_decisions([float(r[6])], m, pn, pc, cf, nf, rw)
        assert int(forced[0]) == int(r[7]), r
        assert int(m_row[0]) == int(r[8]), r
        if r[9] == "-":
            assert w_row is None
        else:
            assert int(w_row[0]) == int(r[9]), r
    for key, pts in groups.items():
        m, pn, pc, cf, nf, rw = int(key[0]), *(float(v) for v in key[1:5]), bool(int(key[5]))
        forced, m_row, w_row = orc.gate_decisions([float(p[0]) for p in pts], m, pn, pc, cf, nf,
                                                  rw)
        np.testing.assert_array_equal(forced, [int(p[1]) for p in pts])
        np.testing.assert_array_equal(m_row, [int(p[2]) for p in pts])
        # budgets only: the same draws and weights, nothing forced
        f2, m2, w2 = orc.gate_decisions([float(p[0]) for p in pts], m, pn, pc, cf, nf, rw,
                                        by_degree=True)
        assert not f2.any()
        np.testing.assert_array_equal(m2, m_row)
        if rw:
            np.testing.assert_array_equal(w2, w_row)


def test_uniform_balls_recovery_improves_with_n(orc):
    """Theorem 1 / Figure 1: with s ~ 20 ln n / n the sampled graph recovers
    well-separated clusters once n is large enough; on three uniform balls the
    oracle's ARI against the generating ball rises to 1."""
    aris = []
    for n in (200, 3000):
        x, truth = datagen.uniform_balls(n, seed=1)
        m = int(math.ceil(20 * math.log(n)))
        r = orc.cluster(x, 0.5, seed=1, m=m, min_pts=2)
        aris.append(orc.ari(r["labels"], truth))
    assert aris[-1] > 0.99
    assert aris[-1] >= aris[0]
