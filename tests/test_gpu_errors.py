"""Status codes across the C ABI: invalid arguments are rejected before any
launch, injected allocation failures surface as SNG_ENOMEM without leaking,
and the library keeps working afterwards."""
import os

import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2006_06743_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("field,value", [("eps", 0.0), ("eps", float("nan")), ("min_pts", 0),
                                         ("s", 0.0), ("s", 1.5), ("band_rel", -1.0),
                                         ("map_group", 3), ("map_block", 48),
                                         ("degree_mode", 3)])
def test_invalid_params_rejected(field, value):
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(100, 3, seed=0)).cuda()
    p = sng.Params(eps=0.1, min_pts=3, s=0.1)
    setattr(p, field, value)
    before = sng.launch_count()
    with pytest.raises(sng.SngError) as e:
        sng.cluster(x, p)
    assert e.value.status == sng.SNG_EINVAL
    assert sng.launch_count() == before


def test_draw_count_limit():
    """m within 1024 of 2^31 would overflow the gather's 32-bit draw index:
    rejected before any launch, like SAMPLE_ALL beyond it."""
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(100, 3, seed=0)).cuda()
    before = sng.launch_count()
    with pytest.raises(sng.SngError) as e:
        sng.cluster(x, sng.Params(eps=0.1, min_pts=3, m=2**31 - 1000))
    assert e.value.status == sng.SNG_EINVAL
    assert sng.launch_count() == before


def test_invalid_shapes_rejected():
    torch, sng = need_gpu()
    x = torch.zeros((1, 3), device="cuda")
    with pytest.raises(sng.SngError):
        sng.cluster(x, sng.Params(eps=0.1, min_pts=1, m=1))
    x = torch.zeros((10, 5000), device="cuda")
    with pytest.raises(sng.SngError):
        sng.cluster(x, sng.Params(eps=0.1, min_pts=1, m=1))


def test_injected_alloc_failure_no_leak():
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(5000, 8, seed=3)).cuda()
    p = sng.Params(eps=0.3, min_pts=4, m=64, seed=1)
    ref, _ = sng.cluster(x, p)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 3, 6):
        os.environ["SNG_FAULT_ALLOC"] = str(k)
        try:
            with pytest.raises(sng.SngError) as e:
                sng.cluster(x, p)
            assert e.value.status == sng.SNG_ENOMEM
        finally:
            del os.environ["SNG_FAULT_ALLOC"]
        torch.cuda.synchronize()
    got, _ = sng.cluster(x, p)
    assert torch.equal(got, ref)
    torch.cuda.synchronize()
    # the stream-ordered pool keeps its blocks; nothing beyond it is retained
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


def test_bounded_loops_report_timeout_and_context_survives():
    """Every union-find loop is bounded; forcing the bound down to one step
    (host-side, through SNG_LOOP_LIMIT) makes the device give up, record it in
    the status word and return.  The call reports SNG_ETIMEOUT, nothing
    faults, and the next call with the normal bound is exact again."""
    torch, sng = need_gpu()
    x = torch.from_numpy(datagen.random_points(20_000, 3, seed=9)).cuda()
    p = sng.Params(eps=0.2, min_pts=4, m=64, seed=3)
    ref, st = sng.cluster(x, p)
    assert st["clusters"] >= 1 and st["cores"] > 1000
    os.environ["SNG_LOOP_LIMIT"] = "1"
    try:
        with pytest.raises(sng.SngError) as e:
            sng.cluster(x, p)
        assert e.value.status == sng.SNG_ETIMEOUT
        assert "bounded" in sng.last_error()
    finally:
        del os.environ["SNG_LOOP_LIMIT"]
    again, _ = sng.cluster(x, p)
    assert torch.equal(again, ref)
