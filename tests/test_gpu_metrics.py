"""The clustering scores on the device (adjusted Rand index and adjusted
mutual information, the two scores of the paper's Section 5) against the FP64
oracle on the same labelings.

Tolerances: MI and the entropies are sums of n-term FP64 expressions whose
summation order differs (atomics), relative 1e-12.  The expected MI takes each
hypergeometric mode probability from nine log-gamma values of size up to
n log n that cancel down to log P, on both sides, so it carries a relative
error of about n log(n) 2^-52 times a few ulps (below 1e-8 for n <= 1e6):
relative 1e-7.  The score then differs by at most that error over its
normaliser: absolute 1e-8."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu

AVERAGES = ("min", "geometric", "arithmetic", "max")


def _labels(rng, n, ka, kb, agree):
    a = rng.integers(-1, ka, n).astype(np.int32)
    b = np.where(rng.random(n) < agree, a % max(kb, 1), rng.integers(-1, kb, n)).astype(np.int32)
    return a, b


def _check(orc, sng, torch, a, b, average):
    got = sng.ami(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), average)
    want = orc.ami(a, b, average)
    for k in ("mi", "h_a", "h_b"):
        assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-14), k
    assert got["emi"] == pytest.approx(want["emi"], rel=1e-7, abs=1e-13)
    assert got["ami"] == pytest.approx(want["ami"], abs=1e-8)
    assert got["clusters_a"] == np.unique(a).size
    assert got["clusters_b"] == np.unique(b).size
    return got


@pytest.mark.parametrize("average", AVERAGES)
@pytest.mark.parametrize("seed,n,ka,kb,agree", [(0, 2, 1, 1, 0.5), (1, 7, 3, 2, 0.5),
                                                (2, 1000, 5, 8, 0.8), (3, 20_000, 30, 20, 0.6),
                                                (4, 1200, 400, 300, 0.5),
                                                (5, 200_000, 100, 120, 0.9)])
def test_ami_matches_oracle(orc, average, seed, n, ka, kb, agree):
    torch, sng = need_gpu()
    a, b = _labels(np.random.default_rng(seed), n, ka, kb, agree)
    _check(orc, sng, torch, a, b, average)


def test_ami_special_cases(orc):
    torch, sng = need_gpu()
    n = 120   # the oracle sums every (cluster, cluster) pair: n^2 for singletons
    cases = [(np.zeros(n), np.full(n, 4)), (np.arange(n), np.arange(n)[::-1]),
             (np.zeros(n), np.arange(n) % 7), (np.arange(n) % 9, (np.arange(n) % 9) * 3 - 1)]
    for a, b in cases:
        a, b = a.astype(np.int32), b.astype(np.int32)
        for average in AVERAGES:
            got = _check(orc, sng, torch, a, b, average)
            assert got["ami"] in (0.0, 1.0) or abs(got["ami"] - 1.0) < 1e-12


def test_ami_of_sng_clustering_against_ground_truth(orc):
    """The score the paper reports: SNG-DBSCAN labels (noise one label) against
    the generating mixture components."""
    torch, sng = need_gpu()
    x, truth = datagen.gaussian_mixture(100_000, 8, k=20, noise_frac=0.02, seed=3,
                                        return_truth=True)
    p = sng.Params(eps=2.5, min_pts=10, s=0.01, seed=1)
    labels, _ = sng.cluster(torch.from_numpy(x).cuda(), p)
    lab = labels.cpu().numpy()
    got = _check(orc, sng, torch, lab, truth.astype(np.int32), "arithmetic")
    assert got["clusters_a"] > 1


def test_ami_rejects_bad_labels():
    torch, sng = need_gpu()
    a = torch.zeros(10, dtype=torch.int32, device="cuda")
    b = torch.full((10,), 10, dtype=torch.int32, device="cuda")
    with pytest.raises(sng.SngError) as e:
        sng.ami(a, b)
    assert e.value.status == sng.SNG_EINVAL
