"""BF16 form: coordinates stored as bfloat16 (16-byte loads of 8 values),
FP32 arithmetic, FP64 recheck from the FP32 master copy inside the band.

Two checks.  (1) When the master copy holds exactly the BF16 values, the FP32
screen is certified and the result must equal the FP64 oracle bit for bit.
(2) With a true FP32 master, every decision inside the band equals the
oracle's; decisions outside it may differ only where BF16 quantisation moves
d^2 across eps^2, and those are counted (the edge-decision error)."""
import math

import numpy as np
import pytest

from gpu_util import BAND_BF16, need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def _bf16_pair(torch, x):
    bits = datagen.bf16_round(x)
    xb = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    return xb, datagen.bf16_to_f32(bits)


@pytest.mark.parametrize("n,d", [(3000, 128), (2000, 64), (1500, 8), (1200, 5), (900, 130)])
def test_bf16_exact_when_master_is_bf16(orc, n, d):
    torch, sng = need_gpu()
    x = datagen.random_points(n, d, seed=d)
    xb, xq = _bf16_pair(torch, x)
    master = torch.from_numpy(xq).cuda()
    eps = float(np.float32(0.12 * math.sqrt(d)))
    p = sng.Params(eps=eps, min_pts=4, m=200, seed=d)
    g = sng.build_graph(xb, p, x_master=master)
    rp, col, band_pairs, _ = orc.build_rows(xq, eps, p.seed, 200, band_rel=BAND_BF16)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    assert g["stats"]["band_pairs"] == band_pairs
    labels, st = sng.cluster(xb, p, x_master=master)
    r = orc.cluster(xq, eps, p.seed, 200, 4, band_rel=BAND_BF16)
    np.testing.assert_array_equal(labels.cpu().numpy(), r["labels"])


def test_bf16_decision_errors_are_quantisation_only(orc):
    torch, sng = need_gpu()
    n, d, m = 4000, 128, 300
    x = datagen.sphere_embeddings(n, d, 20, 0.0375, seed=4)
    xb, xq = _bf16_pair(torch, x)
    eps = 0.6
    p = sng.Params(eps=eps, min_pts=8, m=m, seed=1)
    g = sng.build_graph(xb, p, x_master=torch.from_numpy(x).cuda())
    got_rp, got_col = g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()
    rp, col, _, _ = orc.build_rows(x, eps, p.seed, m, band_rel=BAND_BF16)
    parts = orc.partners(p.seed, n, 0, n, m)
    eps2 = float(np.float32(eps)) ** 2
    x64, q64 = x.astype(np.float64), xq.astype(np.float64)
    wrong = 0
    for i in range(n):
        a = set(got_col[got_rp[i]:got_rp[i + 1]].tolist())
        b = set(col[rp[i]:rp[i + 1]].tolist())
        for q in a ^ b:
            d2_true = ((x64[i] - x64[q]) ** 2).sum()
            d2_q = ((q64[i] - q64[q]) ** 2).sum()
            # outside the band on the BF16 side, and on the other side of eps^2
            assert abs(d2_q - eps2) > BAND_BF16 * eps2 * 0.999
            assert (d2_q <= eps2) != (d2_true <= eps2)
            wrong += 1
    kept = len(col)
    assert kept > 1000
    assert wrong <= 0.01 * kept, (wrong, kept)


def test_bf16_clustering_close_to_plain():
    torch, sng = need_gpu()
    n, d = 60_000, 128
    x = datagen.sphere_embeddings(n, d, 100, 0.0375, seed=7)
    xb, _ = _bf16_pair(torch, x)
    xf = torch.from_numpy(x).cuda()
    p = sng.Params(eps=0.6, min_pts=8, m=400, seed=3)
    lf, sf = sng.cluster(xf, p)
    lb, sb = sng.cluster(xb, p, x_master=xf)
    assert sng.ari(lb, lf) >= 0.99
    assert sf["clusters"] > 10
