"""The simulation of the paper's Figure 1 (Section 3) on the GPU: a uniform
mixture of three unit balls in R^3, m = ceil(20 ln n) draws per point (the
caption's sampling rate), eps = 0.5 and MinPts = 2.  Labels equal the
oracle's, and the recovery of the generating balls improves with n as
Theorem 1 states (ARI against the generating ball, computed by the oracle)."""
import math

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_figure1_balls_labels_and_recovery(orc):
    torch, sng = need_gpu()
    aris = []
    for n in (300, 1000, 10_000, 100_000):
        x, truth = datagen.uniform_balls(n, seed=0)
        m = int(math.ceil(20.0 * math.log(n)))
        p = sng.Params(eps=0.5, min_pts=2, m=m, seed=0)
        labels, st = sng.cluster(torch.from_numpy(x).cuda(), p)
        r = orc.cluster(x, 0.5, 0, m, 2, band_rel=BAND_F32)
        got = labels.cpu().numpy()
        np.testing.assert_array_equal(got, r["labels"], err_msg=f"n={n}")
        assert st["queries"] == n * m
        a = orc.ari(got, truth)
        gpu_a = sng.ari(labels, torch.from_numpy(truth.astype(np.int32)).cuda())
        assert abs(gpu_a - a) < 1e-12
        aris.append(a)
    assert all(b >= a for a, b in zip(aris, aris[1:])), aris
    assert aris[0] < 0.99 and aris[-1] > 0.999, aris
