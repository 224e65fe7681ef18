"""Pins of the oracle's similarity neighbourhoods (inner product and cosine
similarity in place of the Euclidean ball; the paper's Section 1 notes the
method needs only similarity queries): exact integer inner products, cosines
with exactly representable quotients, the >= at the threshold, and, with
every pair queried (s = 1), textbook DBSCAN under scikit-learn's cosine metric
and on a precomputed similarity matrix."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2006_06743_gb300 import datagen


def test_dot_exact_on_integers():
    rng = np.random.default_rng(0)
    for d in (1, 3, 64, 200):
        a = rng.integers(-50, 50, d)
        b = rng.integers(-50, 50, d)
        assert oracle.dot(a, b) == float(int(np.dot(a.astype(object), b.astype(object))))


def test_cosine_closed_forms():
    assert oracle.cosine([3, 4], [4, 3]) == 24 / 25          # |a| = |b| = 5
    assert oracle.cosine([2, 3, 6], [6, 2, 3]) == 36 / 49    # |a| = |b| = 7
    assert oracle.cosine([1, 0, 0], [0, 5, 0]) == 0.0
    assert oracle.cosine([2, 0], [7, 0]) == 1.0
    assert oracle.cosine([2, 0], [-7, 0]) == -1.0
    assert math.isnan(oracle.cosine([0, 0, 0], [1, 2, 3]))


def test_threshold_is_inclusive_and_band_counted():
    """Two points whose FP64 cosine is exactly the (float32-representable)
    threshold are joined; a zero vector is joined to nothing."""
    x = np.array([[1, 0], [0.75, math.sqrt(1 - 0.75 ** 2)], [0, 0]], dtype=np.float32)
    tau = float(oracle.cosine(x[0], x[1]))
    assert np.float32(tau) == tau                      # the threshold is representable
    rp, col, band_pairs, _ = oracle.build_rows(x, tau, 0, 2, sample_all=True, band_rel=1e-6,
                                               metric=oracle.METRIC_COSINE)
    assert list(col[rp[0]:rp[1]]) == [1] and list(col[rp[1]:rp[2]]) == [0]
    assert rp[3] == rp[2]                               # the zero vector has no edge
    assert band_pairs == 2


def _tau_clear_of_ties(sim, tau, gap=1e-9):
    off = sim[~np.eye(sim.shape[0], dtype=bool)]
    return np.min(np.abs(off - tau)) > gap


@pytest.mark.parametrize("seed,n,d,k", [(0, 150, 3, 3), (1, 250, 8, 4), (2, 200, 32, 5)])
def test_cosine_sample_all_equals_textbook_dbscan(seed, n, d, k):
    skc = pytest.importorskip("sklearn.cluster")
    x = datagen.random_points(n, d, seed=seed) - 0.5
    xn = x.astype(np.float64)
    xn /= np.linalg.norm(xn, axis=1, keepdims=True)
    sim = xn @ xn.T
    tau = float(np.float32(np.quantile(sim[np.triu_indices(n, 1)], 0.9)))
    assert _tau_clear_of_ties(sim, tau)
    r = oracle.cluster(x, tau, seed=0, m=n - 1, min_pts=k - 1, deg_mode=1, sample_all=True,
                       metric=oracle.METRIC_COSINE)
    db = skc.DBSCAN(eps=1.0 - tau, min_samples=k, metric="cosine", algorithm="brute").fit(x)
    core = np.zeros(n, dtype=np.uint8)
    core[db.core_sample_indices_] = 1
    np.testing.assert_array_equal(r["core"], core)
    np.testing.assert_array_equal(r["labels"] < 0, db.labels_ < 0)
    c = core.astype(bool)
    assert oracle.ari(r["labels"][c], db.labels_[c]) == 1.0


@pytest.mark.parametrize("seed,n,d,k", [(3, 200, 4, 3), (4, 300, 16, 5)])
def test_dot_sample_all_equals_dbscan_on_precomputed_similarity(seed, n, d, k):
    """Inner-product neighbourhoods as a precomputed dissimilarity C - <a, b>
    (self at distance 0, so min_samples = MinPts + 1)."""
    skc = pytest.importorskip("sklearn.cluster")
    x = (datagen.random_points(n, d, seed=seed) - 0.3).astype(np.float32)
    g = x.astype(np.float64) @ x.astype(np.float64).T
    tau = float(np.float32(np.quantile(g[np.triu_indices(n, 1)], 0.85)))
    assert _tau_clear_of_ties(g, tau, 1e-7)
    big = float(np.max(g)) + 1.0
    dis = big - g
    np.fill_diagonal(dis, 0.0)
    r = oracle.cluster(x, tau, seed=0, m=n - 1, min_pts=k - 1, deg_mode=1, sample_all=True,
                       metric=oracle.METRIC_DOT)
    db = skc.DBSCAN(eps=big - tau, min_samples=k, metric="precomputed").fit(dis)
    core = np.zeros(n, dtype=np.uint8)
    core[db.core_sample_indices_] = 1
    np.testing.assert_array_equal(r["core"], core)
    np.testing.assert_array_equal(r["labels"] < 0, db.labels_ < 0)


def test_unit_vectors_cosine_matches_euclidean_ball():
    """For unit vectors |a - b|^2 = 2 - 2 cos(a, b): the cosine graph with
    threshold 1 - eps^2/2 is the Euclidean graph with radius eps (no pair is
    within 1e-9 of the threshold here)."""
    x = datagen.sphere_embeddings(3000, 16, 20, 0.1, seed=5)
    eps = 0.5
    tau = 1.0 - eps * eps / 2.0
    rp_l, col_l, _, _ = oracle.build_rows(x, eps, 3, 200)
    rp_c, col_c, _, _ = oracle.build_rows(x, np.float32(tau), 3, 200,
                                          metric=oracle.METRIC_COSINE)
    np.testing.assert_array_equal(rp_l, rp_c)
    np.testing.assert_array_equal(col_l, col_c)
    assert 0 < col_l.size < 3000 * 200


# ------------------------------------------------------ Manhattan / Chebyshev

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pair_metrics.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b, l1, linf = (f.strip() for f in line.split("|"))
        rows.append((np.array([float(v) for v in a.split(",")], dtype=np.float32),
                     np.array([float(v) for v in b.split(",")], dtype=np.float32),
                     float(l1), float(linf)))
    return rows


def test_pair_metrics_hand_values():
    """The distances worked by hand in tests/golden/pair_metrics.txt, both
    argument orders."""
    rows = _golden_rows()
    assert len(rows) == 7
    for a, b, l1, linf in rows:
        assert oracle.l1(a, b) == l1 and oracle.l1(b, a) == l1
        assert oracle.linf(a, b) == linf and oracle.linf(b, a) == linf


def test_pair_metrics_norm_inequalities_and_scipy():
    """L-inf <= L2 <= L1 <= sqrt(d) L2 and L1 <= d L-inf (from the oracle's own
    Euclidean distance), and the values of scipy's cityblock / chebyshev."""
    dist = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(7)
    for d in (1, 2, 5, 16, 64, 300):
        for _ in range(20):
            a = rng.normal(size=d).astype(np.float32) * np.float32(rng.uniform(0.01, 100))
            b = rng.normal(size=d).astype(np.float32)
            l1, linf = oracle.l1(a, b), oracle.linf(a, b)
            l2 = math.sqrt(oracle.dist2(a, b))
            tol = 1e-12 * (l1 + 1.0)
            assert linf <= l2 + tol and l2 <= l1 + tol
            assert l1 <= math.sqrt(d) * l2 + tol and l1 <= d * linf + tol
            assert abs(l1 - dist.cityblock(a.astype(np.float64), b.astype(np.float64))) <= tol
            assert linf == dist.chebyshev(a.astype(np.float64), b.astype(np.float64))


def test_pair_metrics_nan_and_inf():
    nan, inf = float("nan"), float("inf")
    assert math.isnan(oracle.l1([0.0, nan], [0.0, 0.0]))
    assert math.isnan(oracle.linf([nan, 0.0], [0.0, 5.0]))       # not dropped by the max
    assert math.isnan(oracle.linf([inf], [inf]))                   # inf - inf
    assert oracle.l1([inf, 0.0], [0.0, 0.0]) == inf and oracle.linf([0.0, -inf], [0.0, 1.0]) == inf


@pytest.mark.parametrize("metric,sk_metric", [(oracle.METRIC_L1, "manhattan"),
                                              (oracle.METRIC_LINF, "chebyshev")])
@pytest.mark.parametrize("seed,n,d,k", [(0, 150, 2, 3), (1, 250, 5, 4), (2, 200, 16, 5)])
def test_pair_metrics_sample_all_equal_textbook_dbscan(metric, sk_metric, seed, n, d, k):
    """s = 1 reduces Algorithm 1 to DBSCAN under the same distance:
    scikit-learn's brute-force DBSCAN with that metric gives the same cores,
    the same partition of the cores and the same noise."""
    skc = pytest.importorskip("sklearn.cluster")
    dist = pytest.importorskip("scipy.spatial.distance")
    x = datagen.random_points(n, d, seed=seed)
    dm = dist.squareform(dist.pdist(x.astype(np.float64),
                                    "cityblock" if sk_metric == "manhattan" else sk_metric))
    eps = float(np.float32(np.quantile(dm[np.triu_indices(n, 1)], 0.05)))
    off = dm[~np.eye(n, dtype=bool)]
    assert np.min(np.abs(off - eps)) > 1e-9 * eps            # no pair at the threshold
    r = oracle.cluster(x, eps, seed=0, m=n - 1, min_pts=k - 1, deg_mode=1, sample_all=True,
                       metric=metric)
    db = skc.DBSCAN(eps=eps, min_samples=k, metric=sk_metric, algorithm="brute").fit(
        x.astype(np.float64))
    core = np.zeros(n, dtype=np.uint8)
    core[db.core_sample_indices_] = 1
    np.testing.assert_array_equal(r["core"], core)
    np.testing.assert_array_equal(r["labels"] < 0, db.labels_ < 0)
    c = core.astype(bool)
    assert oracle.ari(r["labels"][c], db.labels_[c]) == 1.0


@pytest.mark.parametrize("metric", [oracle.METRIC_L1, oracle.METRIC_LINF])
def test_pair_metric_threshold_is_inclusive_and_band_counted(metric):
    """Integer grid points at distance exactly eps (an integer) are kept and
    counted in the band."""
    x = np.array([[0, 0], [1, 1], [2, 0], [5, 5]], dtype=np.float32)
    eps = 2.0 if metric == oracle.METRIC_L1 else 1.0
    rp, col, band_pairs, _ = oracle.build_rows(x, eps, 0, 3, sample_all=True, metric=metric)
    got = {(i, int(c)) for i in range(4) for c in col[rp[i]:rp[i + 1]]}
    # L1: (0,1) and (1,2) at 2, (0,2) at 2;  L-inf: (0,1), (1,2) at 1, (0,2) at 2 > 1
    want = {(0, 1), (1, 0), (1, 2), (2, 1)}
    if metric == oracle.METRIC_L1:
        want |= {(0, 2), (2, 0)}
    assert got == want and band_pairs == len(want)
