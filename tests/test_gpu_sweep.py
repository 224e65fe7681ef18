"""Randomised sweep: many small problems (seeded shapes, draw counts,
MinPts, degree definitions, neighbourhood tests, padded strides) through
sng_cluster, each compared with the FP64 oracle label for label and counter
for counter."""
import math

import numpy as np
import pytest

from gpu_util import BAND_F32, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", range(40))
def test_random_problem_matches_oracle(orc, case):
    torch, sng = need_gpu()
    rng = np.random.default_rng(1000 + case)
    n = int(rng.integers(2, 3000))
    d = int(rng.choice([1, 2, 3, 4, 5, 7, 8, 12, 16, 24, 31, 32, 33, 48, 64, 65, 100, 128]))
    m = int(rng.integers(1, 400))
    metric = int(rng.choice([0, 0, 0, 1, 2]))
    deg_mode = int(rng.choice([0, 1, 2]))
    min_pts = int(rng.integers(1, 12))
    x = datagen.random_points(n, d, seed=case) - (0.5 if metric else 0.0)
    x = np.ascontiguousarray(x, dtype=np.float32)
    if metric:
        xd = x.astype(np.float64)
        i, j = rng.integers(0, n, 2000), rng.integers(0, n, 2000)
        s = (xd[i] * xd[j]).sum(1)
        if metric == 2:
            s /= np.linalg.norm(xd[i], axis=1) * np.linalg.norm(xd[j], axis=1) + 1e-300
        eps = float(np.float32(np.quantile(s, rng.uniform(0.8, 0.99))))
    else:
        eps = float(np.float32(rng.uniform(0.05, 0.3) * math.sqrt(d)))
    pad = int(rng.choice([0, 0, 1, 3, 4]))
    buf = torch.full((n, d + pad), float("nan"), dtype=torch.float32, device="cuda")
    buf[:, :d] = torch.from_numpy(x).cuda()
    xg = buf[:, :d]
    p = sng.Params(eps=eps, min_pts=min_pts, m=m, seed=case, metric=metric,
                   degree_mode=deg_mode)
    labels, core, st = sng.cluster(xg, p, want_core=True)
    r = orc.cluster(x, eps, case, m, min_pts, deg_mode=deg_mode, band_rel=BAND_F32,
                    metric=metric)
    np.testing.assert_array_equal(core.cpu().numpy(), r["core"])
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])
    for k in ("kept_edges", "band_pairs", "band_points", "cores", "clusters", "noise"):
        assert st[k] == r[k], (k, st[k], r[k])
