"""The autotuner on a point set larger than 48 MiB, where its candidates
include slice passes and the L2-tiled form: whatever mapping wins, its
labels, core flags and counts equal the default mapping's, and the result is
cached per shape."""
import json

import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_tuned_mapping_gives_the_default_result(tmp_path):
    torch, sng = need_gpu()
    from paper_2006_06743_gb300 import autotune
    n, d = 300_000, 64
    x = torch.from_numpy(datagen.gaussian_mixture(n, d, 50, 0.02, seed=3)).cuda()
    p = sng.Params(eps=8.0, min_pts=10, m=200, seed=4)
    cands = autotune.candidates(x, p)
    assert any(c.get("tiled") for c in cands)
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(x, p, reps=1, budget_s=6.0, cache=cache)
    assert best["tried"] >= 4 and best["gather_ms"] > 0
    assert any(c.get("tiled") for _, c in best["table"]) or not best["mapping"].get("tiled")
    tuned = autotune.apply(p, best)
    l0, c0, s0 = sng.cluster(x, p, want_core=True)
    l1, c1, s1 = sng.cluster(x, tuned, want_core=True)
    assert torch.equal(l0, l1) and torch.equal(c0, c1)
    for k in ("kept_edges", "band_pairs", "cores", "clusters", "noise"):
        assert s0[k] == s1[k], k
    assert bool(s1["map_tiles"]) == bool(best["mapping"].get("tiled"))
    with open(cache) as f:
        assert autotune.key_for(x, p) in json.load(f)
    again = autotune.tune(x, p, cache=cache)          # served from the cache
    assert again["mapping"] == best["mapping"]
