"""Pins of the oracle's adjusted mutual information (the paper's second
clustering score, Section 5, after Vinh, Epps & Bailey 2010): the expected
mutual information against a brute-force average over every permutation of
one labelling, entropies and MI against closed forms, the special cases, and
scikit-learn's implementation where it is installed."""
import itertools
import math

import numpy as np
import pytest

import oracle


def _mi_direct(a, b):
    """MI from the definition with Python dictionaries (independent of the
    oracle's contingency table code)."""
    n = len(a)
    ca, cb, cab = {}, {}, {}
    for u, v in zip(a, b):
        ca[u] = ca.get(u, 0) + 1
        cb[v] = cb.get(v, 0) + 1
        cab[(u, v)] = cab.get((u, v), 0) + 1
    return sum(c / n * math.log(n * c / (ca[u] * cb[v])) for (u, v), c in cab.items())


@pytest.mark.parametrize("a,b", [([0, 0, 1, 1, 1, 2, 2], [0, 1, 1, 0, 2, 2, 2]),
                                 ([0, 0, 0, 0, 1, 1, 1], [0, 0, 1, 1, 2, 2, 3]),
                                 ([5, 5, 5, 5, 5, 9, 9], [-1, -1, 0, 0, 0, 0, 0]),
                                 ([0, 1, 2, 3, 4, 5, 6], [0, 0, 0, 1, 1, 1, 1])])
def test_emi_equals_average_over_all_permutations(a, b):
    """E[MI] under the permutation model is, by definition, the mean MI over
    all n! orderings of one labelling (n = 7: 5040 orderings)."""
    perms = list(itertools.permutations(b))
    brute = sum(_mi_direct(a, p) for p in perms) / len(perms)
    t = oracle._contingency(a, b)
    emi = oracle.expected_mutual_info(t.sum(axis=1), t.sum(axis=0), len(a))
    assert emi == pytest.approx(brute, rel=1e-12, abs=1e-15)


def test_mi_and_entropy_closed_forms():
    a = [0, 0, 1, 1]
    t = oracle._contingency(a, a)
    assert oracle.mutual_info(t) == pytest.approx(math.log(2), rel=1e-15)
    assert oracle.entropy([25, 25, 25, 25], 100) == pytest.approx(math.log(4), rel=1e-15)
    # independent labellings on a product grid: MI = 0 exactly
    a = [i // 3 for i in range(9)]
    b = [i % 3 for i in range(9)]
    assert abs(oracle.mutual_info(oracle._contingency(a, b))) < 1e-15
    rng = np.random.default_rng(1)
    a, b = rng.integers(0, 4, 200), rng.integers(-1, 5, 200)
    assert oracle.mutual_info(oracle._contingency(a, b)) == pytest.approx(_mi_direct(a, b),
                                                                          rel=1e-12)


@pytest.mark.parametrize("average", oracle.AMI_AVERAGES)
def test_ami_special_cases(average):
    rng = np.random.default_rng(2)
    a = rng.integers(-1, 6, 500)
    relabel = np.array([7, 3, 11, 0, 5, 2, 9])[a + 1]
    assert oracle.ami(a, relabel, average)["ami"] == pytest.approx(1.0, abs=1e-12)
    assert oracle.ami(np.zeros(50), np.full(50, 3), average)["ami"] == 1.0
    assert oracle.ami(np.arange(50), np.arange(50)[::-1], average)["ami"] == 1.0
    assert oracle.ami(np.zeros(50), np.arange(50) % 4, average)["ami"] == 0.0


def test_ami_symmetric_and_near_zero_for_independent_labels():
    rng = np.random.default_rng(3)
    a, b = rng.integers(0, 8, 3000), rng.integers(0, 5, 3000)
    r1, r2 = oracle.ami(a, b), oracle.ami(b, a)
    assert r1["ami"] == pytest.approx(r2["ami"], rel=1e-12)
    assert abs(r1["ami"]) < 0.01


@pytest.mark.parametrize("average", oracle.AMI_AVERAGES)
@pytest.mark.parametrize("seed,n,ka,kb", [(0, 100, 3, 4), (1, 2000, 10, 6), (2, 5000, 40, 30),
                                          (3, 800, 2, 200)])
def test_ami_matches_scikit_learn(average, seed, n, ka, kb):
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(seed)
    a = rng.integers(-1, ka, n)
    b = np.where(rng.random(n) < 0.7, a, rng.integers(-1, kb, n))
    want = skm.adjusted_mutual_info_score(a, b, average_method=average)
    assert oracle.ami(a, b, average)["ami"] == pytest.approx(want, rel=1e-9, abs=1e-12)
